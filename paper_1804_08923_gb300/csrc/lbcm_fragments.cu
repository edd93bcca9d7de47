// lbcm_fragments.cu -- fragment analysis of a state (arXiv:1804.08923, Section IV.B: binarise
// the order parameter, connected components, volume, equivalent spherical diameter).
//
// Labelling is union-find over the lattice with lock-free links: every jet node starts as
// its own root, each node unites with its jet neighbours in the backward half of the
// neighbourhood (3 face neighbours, or 13 of the 26), and a union links the larger root under
// the smaller with atomicMin.  Parents only decrease and always stay inside the component, so
// after the unions every component is one tree whose root is its smallest linear node index:
// the labels are canonical (independent of the schedule) and comparable with a sequential
// flood fill.  Volumes come from integer atomics on the root; the roots are compacted in index
// order (per-block counts, one scan, per-block ballots), so the output is deterministic.
#include "lbcm_device.cuh"
#include "lbcm_internal.h"

#include <algorithm>

namespace lbcm {

// Smallest-index root of x (parents only decrease: at most x steps).  Volatile reads: other
// SMs relink parents during the union kernel, and a stale cached parent would only cost retries.
__device__ __forceinline__ int frag_find(const volatile int *p, int x, int limit, int *err) {
    for (int it = 0; it < limit; ++it) {
        const int q = p[x];
        if (q == x) return x;
        x = q;
    }
    *err = 1;
    return x;
}

__device__ __forceinline__ void frag_unite(int *p, int a, int b, int limit, int *err) {
    for (int it = 0; it < limit; ++it) {
        a = frag_find(p, a, limit, err);
        b = frag_find(p, b, limit, err);
        if (a == b) return;
        const int hi = max(a, b), lo = min(a, b);
        const int old = atomicMin(&p[hi], lo);
        if (old == hi) return;  // hi was a root and now hangs under lo
        a = old;                // hi was linked meanwhile: unite its new parent with lo
        b = lo;
    }
    *err = 1;
}

// label[n] = n for jet nodes (phi > 0 of the state's colour densities), -1 otherwise.
template <int S>
__global__ void __launch_bounds__(256) frag_init_kernel(StepArgs a, int *label) {
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < a.NN; n += (long long)gridDim.x * blockDim.x) {
        const Nbr nb(a, (int)(n % a.nx), (int)((n / a.nx) % a.ny), (int)(n / a.plane));
        float rr = 0.0f, rb = 0.0f;
#pragma unroll
        for (int i = 0; i < 27; ++i) {
            const float2 v = stored_pop<S>(a, nb, i);
            rr += v.x;
            rb += v.y;
        }
        // phi > 0  <=>  rho_r / rho_r0 > rho_b / rho_b0 (Eq. (23))
        label[n] = rr * a.inv_rho_r0 > rb * a.inv_rho_b0 ? (int)n : -1;
    }
}

struct FragGeom {
    int nx, ny, nz, periodic_z, conn, wall_x, wall_y;
    long long NN, plane;
};

__global__ void __launch_bounds__(256) frag_union_kernel(FragGeom g, int *label, int *err) {
    const int limit = (int)min(g.NN, (long long)INT32_MAX);
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < g.NN; n += (long long)gridDim.x * blockDim.x) {
        if (label[n] < 0) continue;
        const int x = (int)(n % g.nx), y = (int)((n / g.nx) % g.ny), z = (int)(n / g.plane);
        // backward half of the neighbourhood: dz < 0, or dz = 0 and dy < 0, or dz = dy = 0, dx < 0
        for (int dz = -1; dz <= 0; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    if (dz == 0 && (dy > 0 || (dy == 0 && dx >= 0))) continue;
                    if (g.conn == 6 && abs(dx) + abs(dy) + abs(dz) != 1) continue;
                    int zz = z + dz;
                    if (zz < 0) {
                        if (!g.periodic_z) continue;
                        zz += g.nz;
                    }
                    if ((g.wall_x && (x + dx < 0 || x + dx >= g.nx)) || (g.wall_y && (y + dy < 0 || y + dy >= g.ny)))
                        continue;  // no neighbour across a side wall
                    const int xx = x + dx < 0 ? x + dx + g.nx : (x + dx >= g.nx ? x + dx - g.nx : x + dx);
                    const int yy = y + dy < 0 ? y + dy + g.ny : (y + dy >= g.ny ? y + dy - g.ny : y + dy);
                    const long long m = (long long)zz * g.plane + (long long)yy * g.nx + xx;
                    if (m != n && label[m] >= 0) frag_unite(label, (int)n, (int)m, limit, err);
                }
    }
}

__global__ void __launch_bounds__(256) frag_compress_kernel(FragGeom g, int *label, int *err) {
    const int limit = (int)min(g.NN, (long long)INT32_MAX);
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < g.NN; n += (long long)gridDim.x * blockDim.x)
        if (label[n] >= 0) label[n] = frag_find(label, label[n], limit, err);
}

// count[root] = nodes of the component; touch[root] = 1 if it has a node on z = 0.
__global__ void __launch_bounds__(256) frag_count_kernel(FragGeom g, const int *label, int *count, uint8_t *touch) {
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < g.NN; n += (long long)gridDim.x * blockDim.x) {
        const int r = label[n];
        if (r < 0) continue;
        atomicAdd(&count[r], 1);
        if (n < g.plane) touch[r] = 1;
    }
}

constexpr int kFragBlock = 1024;

// Roots per block of kFragBlock nodes.
__global__ void __launch_bounds__(kFragBlock) frag_block_count_kernel(FragGeom g, const int *label, int *bc) {
    __shared__ int sh[32];
    const long long n = (long long)blockIdx.x * kFragBlock + threadIdx.x;
    const bool root = n < g.NN && label[n] == (int)n;
    const unsigned m = __ballot_sync(0xffffffffu, root);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = __popc(m);
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < kFragBlock / 32; ++w) s += sh[w];
        bc[blockIdx.x] = s;
    }
}

// Exclusive scan of the block counts (one block; chunks of 1024 in order); total in bc[nblk].
__global__ void __launch_bounds__(1024) frag_scan_kernel(const int *bc, long long nblk, long long *boff) {
    __shared__ long long sh[1024];
    long long carry = 0;
    for (long long base = 0; base < nblk; base += 1024) {
        const long long i = base + threadIdx.x;
        const long long v = i < nblk ? bc[i] : 0;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {  // inclusive Hillis-Steele scan
            const long long t = (int)threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
            __syncthreads();
            sh[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < nblk) boff[i] = carry + sh[threadIdx.x] - v;
        const long long tot = sh[1023];
        __syncthreads();
        carry += tot;
    }
    if (threadIdx.x == 0) boff[nblk] = carry;
}

// Roots in index order with their volumes and z = 0 flags.
__global__ void __launch_bounds__(kFragBlock) frag_write_kernel(FragGeom g, const int *label, const int *count,
                                                               const uint8_t *touch, const long long *boff,
                                                               long long *out_root, long long *out_vol,
                                                               uint8_t *out_touch) {
    __shared__ int sh[32];
    const long long n = (long long)blockIdx.x * kFragBlock + threadIdx.x;
    const bool root = n < g.NN && label[n] == (int)n;
    const unsigned m = __ballot_sync(0xffffffffu, root);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = __popc(m);
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < kFragBlock / 32; ++w) {
            const int c = sh[w];
            sh[w] = s;
            s += c;
        }
    }
    __syncthreads();
    if (root) {
        const long long k = boff[blockIdx.x] + sh[warp] + __popc(m & ((1u << lane) - 1u));
        out_root[k] = n;
        out_vol[k] = count[n];
        out_touch[k] = touch[n];
    }
}

static int frag_grid(long long n) {
    long long b = (n + 255) / 256;
    return (int)std::min<long long>(std::max<long long>(b, 1), 152ll * 32);
}

cudaError_t launch_fragments_label(const StepArgs &a, int storage, int connectivity, int *label, int *count,
                                   uint8_t *touch, int *bc, long long *boff, int *err, cudaStream_t s,
                                   long long *launches) {
    FragGeom g{a.nx, a.ny, a.nz, a.bc_zlo == BC_PERIODIC, connectivity, a.wall_x, a.wall_y, a.NN, a.plane};
    if (storage == STORE_FP16)
        frag_init_kernel<STORE_FP16><<<frag_grid(a.NN), 256, 0, s>>>(a, label);
    else if (storage == STORE_FP16_FIT)
        frag_init_kernel<STORE_FP16_FIT><<<frag_grid(a.NN), 256, 0, s>>>(a, label);
    else
        frag_init_kernel<STORE_FP32><<<frag_grid(a.NN), 256, 0, s>>>(a, label);
    frag_union_kernel<<<frag_grid(a.NN), 256, 0, s>>>(g, label, err);
    frag_compress_kernel<<<frag_grid(a.NN), 256, 0, s>>>(g, label, err);
    frag_count_kernel<<<frag_grid(a.NN), 256, 0, s>>>(g, label, count, touch);
    const long long nblk = (a.NN + kFragBlock - 1) / kFragBlock;
    frag_block_count_kernel<<<(unsigned)nblk, kFragBlock, 0, s>>>(g, label, bc);
    frag_scan_kernel<<<1, 1024, 0, s>>>(bc, nblk, boff);
    *launches += 7;
    return cudaGetLastError();
}

cudaError_t launch_fragments_write(const StepArgs &a, int connectivity, const int *label, const int *count,
                                   const uint8_t *touch, const long long *boff, long long *out_root,
                                   long long *out_vol, uint8_t *out_touch, cudaStream_t s, long long *launches) {
    FragGeom g{a.nx, a.ny, a.nz, a.bc_zlo == BC_PERIODIC, connectivity, a.wall_x, a.wall_y, a.NN, a.plane};
    const long long nblk = (a.NN + kFragBlock - 1) / kFragBlock;
    frag_write_kernel<<<(unsigned)nblk, kFragBlock, 0, s>>>(g, label, count, touch, boff, out_root, out_vol, out_touch);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace lbcm
