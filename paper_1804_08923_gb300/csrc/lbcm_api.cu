// lbcm_api.cu -- host side of the C ABI declared in include/lbcm.h: parameter
// validation, device buffers, initial states, macroscopic fields, FP64 colour-mass
// reduction, checkpoints, and the step loop.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "lbcm.h"
#include "lbcm_device.cuh"
#include "lbcm_internal.h"

namespace {

thread_local std::string g_err;

lb_status fail(lb_status s, const std::string &msg) {
    g_err = msg;
    return s;
}

lb_status cuda_fail(cudaError_t e, const char *where) {
    return fail(LB_ECUDA, std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

#define LB_CUDA(call)                                    \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

constexpr int kMassBlocks = 1024;  // fixed first-stage grid: the reduction order never changes
constexpr int kMassThreads = 256;
constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Bytes of one population buffer: FP32 float2[27][NN]; FP16 (either encoding) float2 rest[NN]
// + __half2[26][NN].
size_t pop_buffer_bytes(size_t nn, int storage) {
    return storage != LB_STORE_FP32 ? 8 * nn + 4 * 26 * nn : 8 * 27 * nn;
}

// Bytes of the phase buffer: FP32 float2[NN]; either FP16 encoding two float4[NN] (one per
// population buffer).
size_t phase_buffer_bytes(size_t nn, int storage) {
    return storage == LB_STORE_FP32 ? align_up(8 * nn) : 2 * align_up(16 * nn);
}

struct AuxLayout {
    size_t disc, zin, zout, partial, done, ops, err, total;
};

AuxLayout aux_layout(const lb_grid &g) {
    const size_t plane = (size_t)g.nx * g.ny;
    AuxLayout L;
    size_t off = 0;
    L.disc = off;
    off = align_up(off + plane);
    L.zin = off;
    off = align_up(off + 18 * plane * sizeof(float));
    L.zout = off;
    off = align_up(off + 18 * plane * sizeof(float));
    L.partial = off;
    off = align_up(off + 2 * kMassBlocks * sizeof(double) + 2 * sizeof(double));
    L.done = off;  // fused step kernel: per-plane completion counters, item sequence, wait flag
    off = align_up(off + (size_t)g.nz * sizeof(unsigned long long));
    L.ops = off;
    off = align_up(off + 2 * (size_t)g.nz * sizeof(int2));
    L.err = off;
    off = align_up(off + sizeof(int));
    L.total = off;
    return L;
}

lb_status validate(const lb_grid *g, const lb_params *p) {
    if (!g || !p) return fail(LB_EINVAL, "grid and params must not be NULL");
    if (g->nx < 1 || g->ny < 1 || g->nz < 1) return fail(LB_EINVAL, "lattice extents must be >= 1");
    const long long nn = (long long)g->nx * g->ny * g->nz;
    if (nn >= (1ll << 31)) return fail(LB_EINVAL, "nx*ny*nz must be < 2^31");
    const bool zlo_ok = g->bc_zlo == LB_BC_PERIODIC || g->bc_zlo == LB_BC_FREESLIP || g->bc_zlo == LB_BC_INLET;
    const bool zhi_ok = g->bc_zhi == LB_BC_PERIODIC || g->bc_zhi == LB_BC_FREESLIP || g->bc_zhi == LB_BC_CONVECTIVE;
    if (!zlo_ok || !zhi_ok) return fail(LB_EINVAL, "bc_zlo must be PERIODIC/FREESLIP/INLET, bc_zhi PERIODIC/FREESLIP/CONVECTIVE");
    if ((g->bc_zlo == LB_BC_PERIODIC) != (g->bc_zhi == LB_BC_PERIODIC))
        return fail(LB_EINVAL, "z must be periodic at both ends or at neither");
    if (g->bc_zlo != LB_BC_PERIODIC && g->nz < 2) return fail(LB_EINVAL, "walls need nz >= 2");
    if ((g->bc_x != LB_BC_PERIODIC && g->bc_x != LB_BC_FREESLIP) || (g->bc_y != LB_BC_PERIODIC && g->bc_y != LB_BC_FREESLIP))
        return fail(LB_EINVAL, "bc_x and bc_y must be PERIODIC or FREESLIP");
    if (g->bc_zhi == LB_BC_CONVECTIVE && g->nz < 3) return fail(LB_EINVAL, "convective outflow needs nz >= 3");
    if (!(p->rho_r0 > 0) || !(p->rho_b0 > 0)) return fail(LB_EINVAL, "rho_r0 and rho_b0 must be > 0");
    if (!(p->nu_r > 0) || !(p->nu_b > 0)) return fail(LB_EINVAL, "nu_r and nu_b must be > 0");
    const double gamma = p->rho_r0 / p->rho_b0;
    const double alpha_r = 1.0 - (1.0 - 8.0 / 27.0) / gamma;
    if (!(alpha_r >= 0.0 && alpha_r < 1.0)) return fail(LB_EINVAL, "density ratio gamma must be >= 19/27 (alpha_r in [0,1))");
    if (!(p->sigma >= 0) || !std::isfinite(p->sigma)) return fail(LB_EINVAL, "sigma must be finite and >= 0");
    if (!std::isfinite(p->beta)) return fail(LB_EINVAL, "beta must be finite");
    const double s[7] = {p->s0, p->s1, p->s2b, p->s3, p->s4, p->s5, p->s6};
    for (double v : s)
        if (!(v >= 0.0 && v < 2.0)) return fail(LB_EINVAL, "relaxation rates must lie in [0, 2)");
    if (!(p->eps_grad >= 0) || !std::isfinite(p->eps_grad)) return fail(LB_EINVAL, "eps_grad must be finite and >= 0");
    if (p->storage != LB_STORE_FP32 && p->storage != LB_STORE_FP16 && p->storage != LB_STORE_FP16_FIT)
        return fail(LB_EINVAL, "storage must be LB_STORE_FP32, LB_STORE_FP16 or LB_STORE_FP16_FIT");
    if (p->check_every < 0) return fail(LB_EINVAL, "check_every must be >= 0");
    if (p->alpha_mix != 0 && p->alpha_mix != 1) return fail(LB_EINVAL, "alpha_mix must be 0 or 1");
    if (p->step_kernel != 0 && p->step_kernel != 1) return fail(LB_EINVAL, "step_kernel must be 0 or 1");
    if (g->bc_zlo == LB_BC_INLET) {
        if (!(p->d_in >= 0) || !std::isfinite(p->d_in) || !std::isfinite(p->u_in) || !std::isfinite(p->noise_amp))
            return fail(LB_EINVAL, "inlet parameters must be finite, d_in >= 0");
        for (int m = 0; m < 16; ++m)
            if (!std::isfinite(p->fourier[m])) return fail(LB_EINVAL, "inlet profile coefficients must be finite");
    }
    for (int d = 0; d < 3; ++d)
        if (!std::isfinite(p->g[d])) return fail(LB_EINVAL, "gravity must be finite");
    return LB_OK;
}

}  // namespace

struct lb_ctx {
    lb_grid g;
    lb_params p;
    cudaStream_t stream = nullptr;
    bool owns = false;
    void *bufs[LB_MAX_BUFFERS] = {};
    size_t sizes[LB_MAX_BUFFERS] = {};
    int nbufs = 0;
    void *pop[2] = {nullptr, nullptr};
    float2 *phase = nullptr;               // FP32: (phi, rho) of the current step
    float4 *ph4[2] = {nullptr, nullptr};   // FP16: (phi, rho, rho_r, rho_b) paired with pop[0], pop[1]
    float4 *mom = nullptr;                 // collision moments written and read within a step
    // fused step kernel (both passes in one cooperative launch)
    unsigned long long *fdone = nullptr;
    int2 *fops = nullptr;
    int *ferr = nullptr;
    unsigned long long epoch = 0;          // fused launches so far (done[] counts accumulate)
    int fgrid = 0, fnops = 0, flag = 0;    // grid, item sequence length and plane lag of the sequence
    float *hist[2] = {nullptr, nullptr};
    uint8_t *disc = nullptr;
    float *zin = nullptr, *zout = nullptr;
    double *partial = nullptr;
    int cur = 0, hcur = 0;
    int64_t step = 0;
    bool initialized = false;
    bool half = false;  // lb_step_gather has run, lb_step_collide has not
    long long nn = 0, plane = 0;
    long long launches = 0;
    std::vector<cudaEvent_t> prof_ev;  // 4 events per recorded step
    std::vector<char> prof_fused;      // whether the recorded step ran the fused step kernel
    int prof_cap = 0, prof_used = 0;
    // discrete-adjoint workspace (one device allocation, grown on demand)
    struct {
        void *base = nullptr;
        size_t bytes = 0;
        float2 *ckpt_pop = nullptr, *seg_pop = nullptr, *lp[2] = {}, *lr[2] = {}, *lgb = nullptr, *objph = nullptr;
        float *ckpt_hist = nullptr, *seg_fm[2] = {}, *seg_hist[2] = {}, *lc = nullptr, *li = nullptr, *lh[2] = {};
        float4 *lga = nullptr, *seg_mom[2] = {}, *seg_g4[2] = {};
        float2 *seg_g2[2] = {};
        // a second stream recomputes the next segment while the context's stream steps back
        // through the current one; events order the two
        cudaStream_t s2 = nullptr;
        cudaEvent_t ev_fwd = nullptr, ev_rec[2] = {}, ev_rev[2] = {};
        double *acc_coll = nullptr, *acc_inlet = nullptr, *acc_obj = nullptr, *out = nullptr;
        long long nblk_coll = 0, nblk_inlet = 0;
        int cl = 0;
        bool valid = false;
    } adj;
};

namespace lbcm {

// ------------------------------------------------------------ initial populations
// f_i^k = rho_k [varphi_i(alpha_k) + w_i P(c_i.u, u^2)]  (Eq. (18) per colour, Phi = 0); the
// rest population takes each colour's remainder of the stored moving ones.
struct InitArgs {
    float *hist;
    const float *fr, *fb, *fu;
    int kind, nx, ny, nz;
    float a0, a1, a2, a3, a4, rho_r0, rho_b0, alpha_r, alpha_b, oma_r, oma_b;
};

__device__ __forceinline__ Nbr node_nbr(const StepArgs &a, long long n) {
    return Nbr(a, (int)(n % a.nx), (int)((n / a.nx) % a.ny), (int)(n / a.plane));
}

// Fields (rho_r, rho_b, u) of node n of the initial state.
__device__ __forceinline__ void init_fields_at(const InitArgs &ia, long long n, float &rr, float &rb, float &ux,
                                               float &uy, float &uz) {
    const int nx = ia.nx, ny = ia.ny, nz = ia.nz;
    const long long NN = (long long)nx * ny * nz;
    const int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((long long)nx * ny));
    ux = uy = uz = 0.0f;
    if (ia.kind == LB_INIT_UNIFORM) {
        rr = ia.a0; rb = ia.a1; ux = ia.a2; uy = ia.a3; uz = ia.a4;
    } else if (ia.kind == LB_INIT_DROPLET) {
        // Section III: rho_r = rho_r0/2 [1 - tanh(2(r-R)/W)], rho_b = rho_b0/2 [1 + tanh(...)]
        const float dx = x - 0.5f * (nx - 1), dy = y - 0.5f * (ny - 1), dz = z - 0.5f * (nz - 1);
        const float r = sqrtf(dx * dx + dy * dy + dz * dz);
        const float t = tanhf(2.0f * (r - ia.a0) / ia.a1);
        rr = 0.5f * ia.rho_r0 * (1.0f - t);
        rb = 0.5f * ia.rho_b0 * (1.0f + t);
    } else if (ia.kind == LB_INIT_JET) {
        rr = 0.0f; rb = ia.rho_b0;
    } else {
        rr = ia.fr[n]; rb = ia.fb[n]; ux = ia.fu[n]; uy = ia.fu[NN + n]; uz = ia.fu[2 * NN + n];
    }
}

// FP16: phase entries (phi, rho, rho_r, rho_b) of the initial state, which its populations
// are encoded for.  FP16_FIT: the packed entry of phi, A, rho and the odd fit of the node's own
// initial populations (the same prediction the phase-field pass makes from gathered ones).
template <int S>
__global__ void init_phase_kernel(InitArgs ia, StepArgs sa) {
    const long long NN = (long long)ia.nx * ia.ny * ia.nz;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < NN; n += (long long)gridDim.x * blockDim.x) {
        float rr, rb, ux, uy, uz;
        init_fields_at(ia, n, rr, rb, ux, uy, uz);
        const float ph = order_parameter(rr, rb, sa.inv_rho_r0, sa.inv_rho_b0);
        if constexpr (S == STORE_FP16) {
            sa.ph_cur[n] = make_float4(ph, rr + rb, rr, rb);
        } else {
            const float usq = ux * ux + uy * uy + uz * uz;
            float fr[27], fb[27];
#pragma unroll
            for (int i = 0; i < 27; ++i) {
                const float cu = (float)cx(i) * ux + (float)cy(i) * uy + (float)cz(i) * uz;
                const float pw = wgt(i) * eq_poly(cu, usq);
                fr[i] = rr * (varphi(i, ia.alpha_r, ia.oma_r) + pw);
                fb[i] = rb * (varphi(i, ia.alpha_b, ia.oma_b) + pw);
            }
            sa.ph_cur[n] = pack_fit_entry(ph, rr + rb, fit_even(sa, rr, rb, ph), fit_odd_fp8(sa, fr, fb));
        }
    }
}

template <int S>
__global__ void init_kernel(InitArgs ia, StepArgs sa) {
    const long long NN = sa.NN;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < NN; n += (long long)gridDim.x * blockDim.x) {
        float rr, rb, ux, uy, uz;
        init_fields_at(ia, n, rr, rb, ux, uy, uz);
        const Nbr nb = node_nbr(sa, n);
        const float usq = ux * ux + uy * uy + uz * uz;
        MassAcc sr, sb;
        const bool top = nb.zo[1] == (ia.nz - 1) * (int)sa.plane;
        const long long h = nb.pxy, P = sa.plane;
#pragma unroll
        for (int i = 1; i < 27; ++i) {
            const float cu = (float)cx(i) * ux + (float)cy(i) * uy + (float)cz(i) * uz;
            const float pw = wgt(i) * eq_poly(cu, usq);
            const float2 f = make_float2(rr * (varphi(i, ia.alpha_r, ia.oma_r) + pw),
                                         rb * (varphi(i, ia.alpha_b, ia.oma_b) + pw));
            const float2 d = store_pop<S>(sa, i, (int)n, f, dest_shift<S>(sa, nb, i));
            sr.add(i, d.x);
            sb.add(i, d.y);
            if (top) {
                ia.hist[(long long)i * P + h] = d.x;
                ia.hist[(long long)(27 + i) * P + h] = d.y;
            }
        }
        const float2 f0 = make_float2(rr - sr.s, rb - sb.s);
        store_pop<S>(sa, 0, (int)n, f0, no_shift());
        if (top) {
            ia.hist[h] = f0.x;
            ia.hist[27 * P + h] = f0.y;
        }
    }
}

// ------------------------------------------------------------------- fields
struct FieldOut {
    float *o[LB_NFIELDS];
};

template <int S>
__global__ void fields_kernel(StepArgs sa, FieldOut fo, float gx, float gy, float gz) {
    const long long NN = sa.NN;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < NN; n += (long long)gridDim.x * blockDim.x) {
        const Nbr nb = node_nbr(sa, n);
        MassAcc mr, mb;
        float jx = 0.0f, jy = 0.0f, jz = 0.0f;
#pragma unroll
        for (int i = 0; i < 27; ++i) {
            const float2 v = stored_pop<S>(sa, nb, i);
            mr.add(i, v.x);
            mb.add(i, v.y);
            if (cx(i) != 0) jx += cx(i) * (v.x + v.y);
            if (cy(i) != 0) jy += cy(i) * (v.x + v.y);
            if (cz(i) != 0) jz += cz(i) * (v.x + v.y);
        }
        const float rr = mr.total(), rb = mb.total();
        const float rho = rr + rb;
        const float phi = order_parameter(rr, rb, sa.inv_rho_r0, sa.inv_rho_b0);
        const float fc = rho - sa.rho_b0;
        if (fo.o[LB_FIELD_RHO_R]) fo.o[LB_FIELD_RHO_R][n] = rr;
        if (fo.o[LB_FIELD_RHO_B]) fo.o[LB_FIELD_RHO_B][n] = rb;
        if (fo.o[LB_FIELD_PHI]) fo.o[LB_FIELD_PHI][n] = phi;
        if (fo.o[LB_FIELD_UX]) fo.o[LB_FIELD_UX][n] = (jx - 0.5f * fc * gx) / rho;
        if (fo.o[LB_FIELD_UY]) fo.o[LB_FIELD_UY][n] = (jy - 0.5f * fc * gy) / rho;
        if (fo.o[LB_FIELD_UZ]) fo.o[LB_FIELD_UZ][n] = (jz - 0.5f * fc * gz) / rho;
        if (fo.o[LB_FIELD_P]) {
            const float oma = sa.alpha_mix ? (rr * sa.oma_r + rb * sa.oma_b) / rho
                                           : 0.5f * (1.0f + phi) * sa.oma_r + 0.5f * (1.0f - phi) * sa.oma_b;
            fo.o[LB_FIELD_P][n] = rho * 9.0f * oma / 19.0f;  // Eq. (26)
        }
    }
}

// Decoded populations of colour k in the canonical layout out[i][n] (27 x NN floats).
template <int S>
__global__ void canonical_kernel(StepArgs sa, int k, float *__restrict__ out) {
    const long long NN = sa.NN;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < NN; n += (long long)gridDim.x * blockDim.x) {
        const Nbr nb = node_nbr(sa, n);
#pragma unroll
        for (int i = 0; i < 27; ++i) {
            const float2 v = stored_pop<S>(sa, nb, i);
            out[(long long)i * NN + n] = k == 0 ? v.x : v.y;
        }
    }
}

// ------------------------------------------------------------- FP64 colour mass
// Stage 1: block b of colour k adds, in FP64 and a fixed order, every population of its
// fixed node range, reduces the block by warp shuffles and writes one partial.  Stage 2:
// one block adds the partials in a fixed tree order.
__global__ void __launch_bounds__(kMassThreads) mass_partial_kernel(const float *__restrict__ pop, long long NN,
                                                                    double *__restrict__ partial) {
    const int k = blockIdx.y;
    const long long per = (NN + gridDim.x - 1) / gridDim.x;
    const long long n0 = blockIdx.x * per, n1 = min(NN, n0 + per);
    double acc = 0.0;
    for (long long n = n0 + threadIdx.x; n < n1; n += blockDim.x) {
#pragma unroll
        for (int i = 0; i < 27; ++i) acc += (double)__ldg(pop + (long long)(27 * k + i) * NN + n);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ double warp_sums[kMassThreads / 32];
    if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kMassThreads / 32; ++w) t += warp_sums[w];
        partial[k * gridDim.x + blockIdx.x] = t;
    }
}

// Same first stage over a context's own population storage (decoded).
template <int S>
__global__ void __launch_bounds__(kMassThreads) mass_partial_store_kernel(StepArgs sa, long long nb, long long ne,
                                                                          double *__restrict__ partial) {
    const int k = blockIdx.y;
    const long long per = (ne - nb + gridDim.x - 1) / gridDim.x;
    const long long n0 = nb + blockIdx.x * per, n1 = min(ne, n0 + per);
    double acc = 0.0;
    for (long long n = n0 + threadIdx.x; n < n1; n += blockDim.x) {
        const Nbr nb = node_nbr(sa, n);
#pragma unroll
        for (int i = 0; i < 27; ++i) {
            const float2 v = stored_pop<S>(sa, nb, i);
            acc += (double)(k == 0 ? v.x : v.y);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ double warp_sums[kMassThreads / 32];
    if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kMassThreads / 32; ++w) t += warp_sums[w];
        partial[k * gridDim.x + blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(1024) mass_final_kernel(const double *__restrict__ partial, int nblocks,
                                                          double *__restrict__ out) {
    __shared__ double s[1024];
    for (int k = 0; k < 2; ++k) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += partial[k * nblocks + b];
        s[threadIdx.x] = v;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[k] = s[0];
        __syncthreads();
    }
}

// Scratch of lb_mass_noalloc: first-stage partials of both colours, then the two results.
static __device__ __align__(256) double g_mass_noalloc_scratch[2 * LB_MASS_NOALLOC_MAX_BLOCKS + 2];

}  // namespace lbcm

namespace {

using namespace lbcm;


// Inlet disc membership for the current d_in, and cleared boundary planes.
lb_status upload_disc(lb_ctx *c) {
    const lb_grid &g = c->g;
    // inlet disc membership, decided in FP64 on the host:
    // (2x - (nx-1))^2 + (2y - (ny-1))^2 < D^2  <=>  (x - x_c)^2 + (y - y_c)^2 < (D/2)^2
    std::vector<uint8_t> disc((size_t)c->plane, 0);
    if (g.bc_zlo == LB_BC_INLET) {
        for (int y = 0; y < g.ny; ++y)
            for (int x = 0; x < g.nx; ++x) {
                const double dx = 2.0 * x - (g.nx - 1), dy = 2.0 * y - (g.ny - 1);
                disc[(size_t)y * g.nx + x] = dx * dx + dy * dy < c->p.d_in * c->p.d_in;
            }
    }
    LB_CUDA(cudaMemcpyAsync(c->disc, disc.data(), disc.size(), cudaMemcpyHostToDevice, c->stream));
    LB_CUDA(cudaMemsetAsync(c->zin, 0, 18 * c->plane * sizeof(float), c->stream));
    LB_CUDA(cudaMemsetAsync(c->zout, 0, 18 * c->plane * sizeof(float), c->stream));
    LB_CUDA(cudaStreamSynchronize(c->stream));
    return LB_OK;
}

lb_status setup_ctx(lb_ctx *c) {
    const lb_grid &g = c->g;
    c->nn = (long long)g.nx * g.ny * g.nz;
    c->plane = (long long)g.nx * g.ny;
    const size_t hist_bytes = (size_t)54 * c->plane * sizeof(float);
    c->pop[0] = c->bufs[0];
    c->pop[1] = c->bufs[1];
    if (c->p.storage != LB_STORE_FP32) {
        const size_t b4 = align_up(16 * (size_t)c->nn);
        c->ph4[0] = (float4 *)c->bufs[2];
        c->ph4[1] = (float4 *)((char *)c->bufs[2] + b4);
    } else {
        c->phase = (float2 *)c->bufs[2];
    }
    c->hist[0] = (float *)c->bufs[3];
    c->hist[1] = (float *)((char *)c->bufs[3] + align_up(hist_bytes));
    const AuxLayout L = aux_layout(g);
    char *aux = (char *)c->bufs[4];
    c->disc = (uint8_t *)(aux + L.disc);
    c->zin = (float *)(aux + L.zin);
    c->zout = (float *)(aux + L.zout);
    c->partial = (double *)(aux + L.partial);
    c->mom = (float4 *)c->bufs[5];
    c->fdone = (unsigned long long *)(aux + L.done);
    c->fops = (int2 *)(aux + L.ops);
    c->ferr = (int *)(aux + L.err);
    LB_CUDA(cudaMemsetAsync(c->fdone, 0, (size_t)g.nz * sizeof(unsigned long long), c->stream));
    LB_CUDA(cudaMemsetAsync(c->ferr, 0, sizeof(int), c->stream));
    return upload_disc(c);
}

StepArgs make_args(const lb_ctx *c) {
    const lb_grid &g = c->g;
    const lb_params &p = c->p;
    StepArgs a{};
    a.pin = c->pop[c->cur];
    a.pout = c->pop[c->cur ^ 1];
    a.phase = c->phase;
    a.ph_prev = c->ph4[c->cur];
    a.ph_cur = c->ph4[c->cur ^ 1];
    a.mom = c->mom;
    a.hist_in = c->hist[c->hcur];
    a.hist_out = c->hist[c->hcur ^ 1];
    a.zin = c->zin;
    a.zout = c->zout;
    a.disc = c->disc;
    a.NN = c->nn;
    a.plane = c->plane;
    a.nx = g.nx; a.ny = g.ny; a.nz = g.nz;
    a.bc_zlo = g.bc_zlo; a.bc_zhi = g.bc_zhi;
    a.wall_x = g.bc_x == LB_BC_FREESLIP;
    a.wall_y = g.bc_y == LB_BC_FREESLIP;
    a.rho_r0 = (float)p.rho_r0; a.rho_b0 = (float)p.rho_b0;
    a.inv_rho_r0 = (float)(1.0 / p.rho_r0); a.inv_rho_b0 = (float)(1.0 / p.rho_b0);
    const double alpha_b = 8.0 / 27.0;
    a.alpha_b = (float)alpha_b;
    a.alpha_mix = p.alpha_mix;
    a.alpha_r = (float)(1.0 - (1.0 - alpha_b) / (p.rho_r0 / p.rho_b0));
    a.oma_r = (float)((1.0 - alpha_b) / (p.rho_r0 / p.rho_b0));
    a.oma_b = (float)(1.0 - alpha_b);
    a.inv_nu_r = (float)(1.0 / p.nu_r); a.inv_nu_b = (float)(1.0 / p.nu_b);
    a.sigma = (float)p.sigma; a.beta = (float)p.beta;
    a.eps2 = (float)(p.eps_grad * p.eps_grad);
    a.gx = (float)p.g[0]; a.gy = (float)p.g[1]; a.gz = (float)p.g[2];
    a.s0 = (float)p.s0; a.s1 = (float)p.s1; a.s2b = (float)p.s2b; a.s3 = (float)p.s3;
    a.s4 = (float)p.s4; a.s5 = (float)p.s5; a.s6 = (float)p.s6;
    a.u_in = (float)p.u_in; a.noise_amp = (float)p.noise_amp;
    a.xc = (float)(0.5 * (g.nx - 1)); a.yc = (float)(0.5 * (g.ny - 1));
    // FP16 shift weights varphi_i(alpha_k) by speed class (Eq. (20)), one rounding
    const double kq[4] = {0.0, 2.0 / 19.0, 1.0 / 38.0, 1.0 / 152.0};
    const double alpha_r = 1.0 - (1.0 - alpha_b) / (p.rho_r0 / p.rho_b0);
    for (int q = 0; q < 4; ++q) {
        a.shift_r[q] = (float)(kq[q] * (1.0 - alpha_r));
        a.shift_b[q] = (float)(kq[q] * (1.0 - alpha_b));
    }
    // FP16_FIT scales, powers of two tied to the density scale: S_h = 2^floor(log2(1024 /
    // rho_max)) keeps |S_h h| far below the FP16 maximum for |h| up to 64 rho_max while moving
    // the small deviations of a resting fluid out of the subnormal range; S_v = 2^round(log2(64 /
    // rho_max)) maps odd fits up to 7 rho_max (3 rho u for u < 2) into the e4m3 range.
    const double rho_max = std::max(p.rho_r0, p.rho_b0);
    const int eh = std::min(60, std::max(-60, (int)std::floor(std::log2(1024.0 / rho_max))));
    const int ev = std::min(60, std::max(-60, (int)std::lround(std::log2(64.0 / rho_max))));
    a.dev_scale = std::ldexp(1.0f, eh);
    a.inv_dev_scale = std::ldexp(1.0f, -eh);
    a.v_scale = std::ldexp(1.0f, ev);
    const double wq[4] = {8.0 / 27.0, 2.0 / 27.0, 1.0 / 54.0, 1.0 / 216.0};
    for (int q = 0; q < 4; ++q) {
        a.wv[q] = (float)std::ldexp(wq[q], -ev);
        // the prediction's constants in half precision (k_q of Eq. (20) and w_q / S_v)
        const float k = (float)kq[q];
        a.kqh[q] = __floats2half2_rn(k, k);
        a.wvh[q] = __floats2half2_rn(a.wv[q], a.wv[q]);
    }
    for (int m = 0; m < 16; ++m) a.fourier[m] = (float)p.fourier[m];
    a.seed = p.seed;
    a.step = c->step;
    return a;
}

// Step arguments describing the current state for diagnostics: pin = the current
// populations, ph_cur = the phase entries they were encoded for (FP16).
StepArgs state_args(const lb_ctx *c) {
    StepArgs a = make_args(c);
    a.ph_cur = c->ph4[c->cur];
    a.ph_prev = c->ph4[c->cur];
    return a;
}

// FP64 colour masses of planes [z0, z1) of the current state (store-aware first stage).
lb_status run_mass(lb_ctx *c, double out[2], int z0 = 0, int z1 = -1) {
    const StepArgs sa = state_args(c);
    if (z1 < 0) z1 = c->g.nz;
    const long long nb = (long long)z0 * c->plane, ne = (long long)z1 * c->plane;
    const dim3 grid(kMassBlocks, 2);
    if (c->p.storage == LB_STORE_FP16)
        mass_partial_store_kernel<STORE_FP16><<<grid, kMassThreads, 0, c->stream>>>(sa, nb, ne, c->partial);
    else if (c->p.storage == LB_STORE_FP16_FIT)
        mass_partial_store_kernel<STORE_FP16_FIT><<<grid, kMassThreads, 0, c->stream>>>(sa, nb, ne, c->partial);
    else
        mass_partial_store_kernel<STORE_FP32><<<grid, kMassThreads, 0, c->stream>>>(sa, nb, ne, c->partial);
    mass_final_kernel<<<1, 1024, 0, c->stream>>>(c->partial, kMassBlocks, c->partial + 2 * kMassBlocks);
    c->launches += 2;
    LB_CUDA(cudaGetLastError());
    LB_CUDA(cudaMemcpyAsync(out, c->partial + 2 * kMassBlocks, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    int err = 0;
    LB_CUDA(cudaMemcpyAsync(&err, c->ferr, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    LB_CUDA(cudaStreamSynchronize(c->stream));
    if (err) {
        cudaMemsetAsync(c->ferr, 0, sizeof(int), c->stream);
        return fail(LB_ETIMEOUT, "a wait of the fused step kernel ran out: the state is not to be trusted");
    }
    return LB_OK;
}

int grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    return (int)std::min<long long>(std::max<long long>(b, 1), 152ll * 64);
}

constexpr uint64_t kMagic = 0x314D43424C4C4231ull;  // "1BLLBCM1"

}  // namespace

extern "C" {

void lb_params_default(lb_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->rho_r0 = 1.0;
    p->rho_b0 = 1.0;
    p->nu_r = p->nu_b = 1.0 / 6.0;
    p->beta = 0.7;
    p->s2b = p->s3 = p->s4 = p->s5 = p->s6 = 1.0;
    p->eps_grad = 1e-6;
    p->storage = LB_STORE_FP32;
}

const char *lb_last_error(void) { return g_err.c_str(); }

lb_status lb_buffer_sizes(const lb_grid *grid, const lb_params *params, size_t *sizes_out, int32_t *n_out) {
    lb_status s = validate(grid, params);
    if (s != LB_OK) return s;
    if (!sizes_out || !n_out) return fail(LB_EINVAL, "sizes_out and n_out must not be NULL");
    const size_t nn = (size_t)grid->nx * grid->ny * grid->nz, plane = (size_t)grid->nx * grid->ny;
    sizes_out[0] = align_up(pop_buffer_bytes(nn, params->storage));
    sizes_out[1] = sizes_out[0];
    sizes_out[2] = phase_buffer_bytes(nn, params->storage);  // phase field
    sizes_out[3] = 2 * align_up(54 * plane * sizeof(float));
    sizes_out[4] = aux_layout(*grid).total;
    sizes_out[5] = align_up(48 * nn);  // collision moments of the step being taken
    *n_out = 6;
    return LB_OK;
}

static lb_status create_common(const lb_grid *grid, const lb_params *params, void *stream, void *const *bufs,
                               const size_t *sizes, int32_t n, bool own, lb_ctx **out) {
    if (!out) return fail(LB_EINVAL, "out must not be NULL");
    size_t need[LB_MAX_BUFFERS];
    int32_t nb = 0;
    lb_status s = lb_buffer_sizes(grid, params, need, &nb);
    if (s != LB_OK) return s;
    lb_ctx *c = new (std::nothrow) lb_ctx();
    if (!c) return fail(LB_ENOMEM, "host allocation of the context failed");
    c->g = *grid;
    c->p = *params;
    c->stream = (cudaStream_t)stream;
    c->owns = own;
    c->nbufs = nb;
    if (own) {
        for (int j = 0; j < nb; ++j) {
            cudaError_t e = cudaMalloc(&c->bufs[j], need[j]);
            if (e != cudaSuccess) {
                for (int q = 0; q < j; ++q) cudaFree(c->bufs[q]);
                delete c;
                (void)cudaGetLastError();
                return fail(LB_ENOMEM, std::string("cudaMalloc of ") + std::to_string(need[j]) + " bytes failed: " +
                                           cudaGetErrorString(e));
            }
            c->sizes[j] = need[j];
        }
    } else {
        if (!bufs || !sizes || n < nb) {
            delete c;
            return fail(LB_EINVAL, "lb_create_with_buffers needs as many buffers as lb_buffer_sizes reports");
        }
        for (int j = 0; j < nb; ++j) {
            if (!bufs[j] || sizes[j] < need[j] || ((uintptr_t)bufs[j] % kAlign) != 0) {
                delete c;
                return fail(LB_EINVAL, "buffer " + std::to_string(j) + " is NULL, too small or not 256-byte aligned");
            }
            c->bufs[j] = bufs[j];
            c->sizes[j] = sizes[j];
        }
    }
    s = setup_ctx(c);
    if (s != LB_OK) {
        lb_destroy(c);
        return s;
    }
    *out = c;
    return LB_OK;
}

lb_status lb_create(const lb_grid *grid, const lb_params *params, void *stream, lb_ctx **out) {
    return create_common(grid, params, stream, nullptr, nullptr, 0, true, out);
}

lb_status lb_create_with_buffers(const lb_grid *grid, const lb_params *params, void *stream, void *const *bufs,
                                 const size_t *sizes, int32_t n, lb_ctx **out) {
    return create_common(grid, params, stream, bufs, sizes, n, false, out);
}

static void free_profile(lb_ctx *c) {
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    c->prof_ev.clear();
    c->prof_cap = c->prof_used = 0;
}

void lb_destroy(lb_ctx *c) {
    if (!c) return;
    free_profile(c);
    if (c->adj.s2) {
        cudaStreamSynchronize(c->adj.s2);
        cudaStreamDestroy(c->adj.s2);
        cudaEventDestroy(c->adj.ev_fwd);
        for (int r = 0; r < 2; ++r) {
            cudaEventDestroy(c->adj.ev_rec[r]);
            cudaEventDestroy(c->adj.ev_rev[r]);
        }
    }
    if (c->adj.base) cudaFree(c->adj.base);
    if (c->owns)
        for (int j = 0; j < c->nbufs; ++j)
            if (c->bufs[j]) cudaFree(c->bufs[j]);
    delete c;
}

lb_status lb_set_params(lb_ctx *c, const lb_params *params) {
    if (!c || !params) return fail(LB_EINVAL, "ctx and params must not be NULL");
    lb_status s = validate(&c->g, params);
    if (s != LB_OK) return s;
    if (params->storage != c->p.storage) return fail(LB_EINVAL, "storage cannot change on an existing context");
    // the FP16 encodings' shift weights and scales derive from rho_r0, rho_b0: a stored state
    // would decode to other populations under new ones
    if (c->p.storage != LB_STORE_FP32 && c->initialized &&
        (params->rho_r0 != c->p.rho_r0 || params->rho_b0 != c->p.rho_b0))
        return fail(LB_EINVAL, "rho_r0 and rho_b0 cannot change on an initialised FP16 context");
    c->p = *params;
    c->adj.valid = false;
    return upload_disc(c);
}

lb_status lb_init(lb_ctx *c, int32_t kind, const double *args, int32_t nargs, const float *rho_r, const float *rho_b,
                  const float *u, int32_t fields_on_device) {
    if (!c) return fail(LB_EINVAL, "ctx must not be NULL");
    float a[5] = {0, 0, 0, 0, 0};
    const float *fr = nullptr, *fb = nullptr, *fu = nullptr;
    switch (kind) {
        case LB_INIT_UNIFORM:
            if (!args || nargs < 5) return fail(LB_EINVAL, "UNIFORM needs args {rho_r, rho_b, ux, uy, uz}");
            for (int j = 0; j < 5; ++j) a[j] = (float)args[j];
            if (!(a[0] >= 0 && a[1] >= 0 && a[0] + a[1] > 0)) return fail(LB_EINVAL, "UNIFORM densities must be >= 0 with a positive sum");
            break;
        case LB_INIT_DROPLET:
            if (!args || nargs < 2 || !(args[0] > 0) || !(args[1] > 0)) return fail(LB_EINVAL, "DROPLET needs args {R > 0, W > 0}");
            a[0] = (float)args[0];
            a[1] = (float)args[1];
            break;
        case LB_INIT_JET:
            break;
        case LB_INIT_FIELDS:
            if (!rho_r || !rho_b || !u) return fail(LB_EINVAL, "FIELDS needs rho_r, rho_b and u");
            break;
        default:
            return fail(LB_EINVAL, "unknown init kind");
    }
    // the state is written into pop[0]; pop[1] stages host fields
    c->cur = 0;
    c->hcur = 0;
    if (kind == LB_INIT_FIELDS) {
        if (fields_on_device) {
            fr = rho_r; fb = rho_b; fu = u;
        } else {
            float *stage = (float *)c->pop[1];
            const size_t nb = (size_t)c->nn * sizeof(float);
            LB_CUDA(cudaMemcpyAsync(stage, rho_r, nb, cudaMemcpyHostToDevice, c->stream));
            LB_CUDA(cudaMemcpyAsync(stage + c->nn, rho_b, nb, cudaMemcpyHostToDevice, c->stream));
            LB_CUDA(cudaMemcpyAsync(stage + 2 * c->nn, u, 3 * nb, cudaMemcpyHostToDevice, c->stream));
            fr = stage; fb = stage + c->nn; fu = stage + 2 * c->nn;
        }
    }
    StepArgs sa = make_args(c);  // cur = 0: the state is written into pop[0] / ph4[0]
    sa.pout = c->pop[0];
    sa.ph_cur = c->ph4[0];
    InitArgs ia{c->hist[0], fr, fb, fu, kind, c->g.nx, c->g.ny, c->g.nz,
                a[0], a[1], a[2], a[3], a[4], sa.rho_r0, sa.rho_b0, sa.alpha_r, sa.alpha_b, sa.oma_r, sa.oma_b};
    if (c->p.storage == LB_STORE_FP16) {
        init_phase_kernel<STORE_FP16><<<grid_for(c->nn, 256), 256, 0, c->stream>>>(ia, sa);
        init_kernel<STORE_FP16><<<grid_for(c->nn, 256), 256, 0, c->stream>>>(ia, sa);
        c->launches += 2;
    } else if (c->p.storage == LB_STORE_FP16_FIT) {
        init_phase_kernel<STORE_FP16_FIT><<<grid_for(c->nn, 256), 256, 0, c->stream>>>(ia, sa);
        init_kernel<STORE_FP16_FIT><<<grid_for(c->nn, 256), 256, 0, c->stream>>>(ia, sa);
        c->launches += 2;
    } else {
        init_kernel<STORE_FP32><<<grid_for(c->nn, 256), 256, 0, c->stream>>>(ia, sa);
        c->launches += 1;
    }
    LB_CUDA(cudaGetLastError());
    if (kind == LB_INIT_FIELDS && !fields_on_device) LB_CUDA(cudaStreamSynchronize(c->stream));
    c->step = 0;
    c->initialized = true;
    c->half = false;
    return LB_OK;
}

// Whether lb_step runs the fused step kernel: selected (step_kernel = 1) and the paper's rates.
static bool use_fused(const lb_ctx *c) {
    const lb_params &p = c->p;
    return p.step_kernel == 1 && p.s3 == 1.0 && p.s4 == 1.0 && p.s5 == 1.0 && p.s6 == 1.0;
}

// A collision item of the fused kernel comes kFusedLeadPct / 100 rounds of the grid's blocks
// after the gather items of the next plane, so that those are usually complete when it starts;
// the moments in flight (held in L2) grow with this lead.  Settable at build time.
#ifndef LBCM_FUSED_LEAD_PCT
#define LBCM_FUSED_LEAD_PCT 100
#endif
constexpr int kFusedLeadPct = LBCM_FUSED_LEAD_PCT;

// Grid of the fused kernel (all blocks resident) and its item sequence: the gathers of plane
// c + lag issued before the collisions of plane c (with periodic z the collisions of plane 0
// need the last plane and come last).  Once per
// context, and again if the grid changes (force switched on or off by lb_set_params).
static lb_status prepare_fused(lb_ctx *c, const StepArgs &a) {
    int occ = 0, dev = 0, sms = 0;
    LB_CUDA(fused_occupancy(a, c->p.storage, &occ));
    LB_CUDA(cudaGetDevice(&dev));
    LB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int nz = c->g.nz;
    const long long T = (long long)((c->g.nx + 31) / 32) * ((c->g.ny + kFusedRows - 1) / kFusedRows);
    const int grid = (int)std::min<long long>((long long)occ * sms, 2 * nz * T);
    if (grid == c->fgrid && c->fnops > 0) return LB_OK;
    c->fgrid = 0;
    if (occ < 1) return LB_OK;  // cannot be resident: two launches
    const bool pz = c->g.bc_zlo == LB_BC_PERIODIC;
    // the collisions of plane c follow the gathers of plane c + 1 by 2 lag - 1 planes of items
    // (the sequence below); lag is chosen so that this is kFusedLeadPct / 100 rounds of the grid
    const long long lead = ((long long)kFusedLeadPct * grid + 99) / 100;
    const int lag = (int)std::max<long long>(1, std::min<long long>(nz - 1, ((lead + T - 1) / T + 2) / 2));
    std::vector<int2> ops;
    int g = 0;
    for (int k = 0; k < nz; ++k) {
        const int cz = pz ? (k + 1) % nz : k;  // periodic: plane 0 last
        const int need = (pz && cz == 0) ? nz - 1 : std::min(nz - 1, cz + lag);
        while (g <= need) ops.push_back(make_int2(0, g++));
        ops.push_back(make_int2(1, cz));
    }
    LB_CUDA(cudaMemcpyAsync(c->fops, ops.data(), ops.size() * sizeof(int2), cudaMemcpyHostToDevice, c->stream));
    LB_CUDA(cudaStreamSynchronize(c->stream));
    c->fnops = (int)ops.size();
    c->flag = lag;
    c->fgrid = grid;
    return LB_OK;
}

// The end of a step: the state now at t+1, and the periodic mass check.
static lb_status finish_step(lb_ctx *c) {
    c->cur ^= 1;
    if (c->g.bc_zhi == LB_BC_CONVECTIVE) c->hcur ^= 1;
    c->step += 1;
    if (c->p.check_every > 0 && c->step % c->p.check_every == 0) {
        double m[2];
        lb_status st = run_mass(c, m);
        if (st != LB_OK) return st;
        if (!std::isfinite(m[0]) || !std::isfinite(m[1]))
            return fail(LB_EUNSTABLE, "non-finite colour mass at step " + std::to_string(c->step));
    }
    return LB_OK;
}

lb_status lb_step_gather(lb_ctx *c) {
    if (!c) return fail(LB_EINVAL, "ctx must not be NULL");
    if (!c->initialized) return fail(LB_ESTATE, "lb_step_gather before lb_init/lb_load");
    if (c->half) return fail(LB_ESTATE, "lb_step_gather twice without lb_step_collide");
    cudaError_t e = launch_step(make_args(c), c->p.storage, c->stream, nullptr, &c->launches, PASS_GATHER);
    if (e != cudaSuccess) return cuda_fail(e, "launch_step (gather)");
    c->half = true;
    return LB_OK;
}

lb_status lb_step_collide(lb_ctx *c) {
    if (!c) return fail(LB_EINVAL, "ctx must not be NULL");
    if (!c->half) return fail(LB_ESTATE, "lb_step_collide without lb_step_gather");
    cudaError_t e = launch_step(make_args(c), c->p.storage, c->stream, nullptr, &c->launches, PASS_COLLIDE);
    if (e != cudaSuccess) return cuda_fail(e, "launch_step (collide)");
    c->half = false;
    return finish_step(c);
}

// Offset, row pitch, row width and row count (bytes) of the parts of plane z of one halo
// kind, in the context's own layout; part 1 is empty (rows = 0) where one part suffices.
struct HaloPart {
    char *base;
    size_t pitch, width, rows;
};
static int halo_parts(lb_ctx *c, int kind, int z, HaloPart (&hp)[2]) {
    const size_t P = (size_t)c->plane, NN = (size_t)c->nn;
    hp[1] = HaloPart{nullptr, 0, 0, 0};
    if (kind == LB_HALO_POPULATIONS) {
        char *pop = (char *)c->pop[c->cur];
        if (c->p.storage == LB_STORE_FP32) {
            hp[0] = HaloPart{pop + (size_t)z * P * 8, NN * 8, P * 8, 27};
        } else {
            hp[0] = HaloPart{pop + (size_t)z * P * 8, P * 8, P * 8, 1};
            hp[1] = HaloPart{pop + NN * 8 + (size_t)z * P * 4, NN * 4, P * 4, 26};
        }
    } else {
        if (c->p.storage == LB_STORE_FP32)
            hp[0] = HaloPart{(char *)(c->phase + (size_t)z * P), P * 8, P * 8, 1};
        else
            hp[0] = HaloPart{(char *)(c->ph4[c->cur ^ 1] + (size_t)z * P), P * 16, P * 16, 1};
    }
    return hp[1].rows ? 2 : 1;
}

static lb_status halo_check(lb_ctx *c, int kind, int z) {
    if (!c) return fail(LB_EINVAL, "ctx must not be NULL");
    if (kind != LB_HALO_POPULATIONS && kind != LB_HALO_PHASE) return fail(LB_EINVAL, "unknown halo kind");
    if (z < 0 || z >= c->g.nz) return fail(LB_EINVAL, "halo plane outside the lattice");
    if (!c->initialized) return fail(LB_ESTATE, "halo copy before lb_init/lb_load");
    if (kind == LB_HALO_POPULATIONS && c->half) return fail(LB_ESTATE, "population halo inside a split step");
    if (kind == LB_HALO_PHASE && !c->half) return fail(LB_ESTATE, "phase halo outside a split step");
    return LB_OK;
}

lb_status lb_halo_bytes(const lb_ctx *c, int32_t kind, size_t *nbytes) {
    if (!c || !nbytes) return fail(LB_EINVAL, "ctx and nbytes must not be NULL");
    const size_t P = (size_t)c->plane;
    const bool fp32 = c->p.storage == LB_STORE_FP32;
    if (kind == LB_HALO_POPULATIONS)
        *nbytes = fp32 ? 216 * P : 112 * P;
    else if (kind == LB_HALO_PHASE)
        *nbytes = fp32 ? 8 * P : 16 * P;
    else
        return fail(LB_EINVAL, "unknown halo kind");
    return LB_OK;
}

static lb_status halo_copy(lb_ctx *c, int kind, int z, char *buf, bool pack, int on_device) {
    HaloPart hp[2];
    const int n = halo_parts(c, kind, z, hp);
    size_t off = 0;
    for (int j = 0; j < n; ++j) {
        const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice
                                           : (pack ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice);
        if (pack)
            LB_CUDA(cudaMemcpy2DAsync(buf + off, hp[j].width, hp[j].base, hp[j].pitch, hp[j].width, hp[j].rows, k,
                                      c->stream));
        else
            LB_CUDA(cudaMemcpy2DAsync(hp[j].base, hp[j].pitch, buf + off, hp[j].width, hp[j].width, hp[j].rows, k,
                                      c->stream));
        off += hp[j].width * hp[j].rows;
    }
    if (!on_device) LB_CUDA(cudaStreamSynchronize(c->stream));
    return LB_OK;
}

lb_status lb_halo_pack(lb_ctx *c, int32_t kind, int32_t z, void *dst, int32_t on_device) {
    lb_status s = halo_check(c, kind, z);
    if (s != LB_OK) return s;
    if (!dst) return fail(LB_EINVAL, "dst must not be NULL");
    return halo_copy(c, kind, z, (char *)dst, true, on_device);
}

lb_status lb_halo_unpack(lb_ctx *c, int32_t kind, int32_t z, const void *src, int32_t on_device) {
    lb_status s = halo_check(c, kind, z);
    if (s != LB_OK) return s;
    if (!src) return fail(LB_EINVAL, "src must not be NULL");
    return halo_copy(c, kind, z, (char *)src, false, on_device);
}

lb_status lb_mass_planes(lb_ctx *c, int32_t z_begin, int32_t z_end, double out[2]) {
    if (!c || !out) return fail(LB_EINVAL, "ctx and out must not be NULL");
    if (!c->initialized) return fail(LB_ESTATE, "lb_mass_planes before lb_init/lb_load");
    if (z_begin < 0 || z_end > c->g.nz || z_begin >= z_end) return fail(LB_EINVAL, "plane range outside the lattice");
    return run_mass(c, out, z_begin, z_end);
}

lb_status lb_step(lb_ctx *c, int64_t n) {
    if (!c) return fail(LB_EINVAL, "ctx must not be NULL");
    if (n < 0) return fail(LB_EINVAL, "n must be >= 0");
    if (!c->initialized) return fail(LB_ESTATE, "lb_step before lb_init/lb_load");
    if (c->half) return fail(LB_ESTATE, "lb_step inside a split step (lb_step_gather without lb_step_collide)");
    for (int64_t s = 0; s < n; ++s) {
        StepArgs a = make_args(c);
        cudaEvent_t *ev = nullptr;
        if (c->prof_used < c->prof_cap) {
            c->prof_fused[c->prof_used] = 0;
            ev = &c->prof_ev[4 * (size_t)c->prof_used++];
        }
        cudaError_t e;
        if (use_fused(c)) {
            lb_status fs = prepare_fused(c, a);
            if (fs != LB_OK) return fs;
        }
        if (c->fgrid > 0 && use_fused(c)) {
            // done[z] grows by the plane's item count in every launch: this launch's target
            const int ty = (c->g.ny + kFusedRows - 1) / kFusedRows;
            const int T = ((c->g.nx + 31) / 32) * ty;
            FusedCtl f{c->fdone, c->fops, c->ferr, (c->epoch + 1) * (unsigned long long)T, c->fnops,
                       (c->g.nx + 31) / 32, ty, c->g.nx % 32 == 0};
            if (ev) c->prof_fused[c->prof_used - 1] = 1;
            e = launch_fused_step(a, c->p.storage, f, c->fgrid, c->stream, ev, &c->launches);
            if (e == cudaSuccess) c->epoch += 1;
        } else {
            e = launch_step(a, c->p.storage, c->stream, ev, &c->launches);
        }
        if (e != cudaSuccess) return cuda_fail(e, "launch_step");
        lb_status st = finish_step(c);
        if (st != LB_OK) return st;
    }
    return LB_OK;
}

int64_t lb_step_count(const lb_ctx *c) { return c ? c->step : -1; }

lb_status lb_fields(lb_ctx *c, uint32_t mask, float *const *outs, int32_t on_device) {
    if (!c || !outs) return fail(LB_EINVAL, "ctx and outs must not be NULL");
    if (!c->initialized) return fail(LB_ESTATE, "lb_fields before lb_init/lb_load");
    if (mask >> LB_NFIELDS) return fail(LB_EINVAL, "unknown field bit in mask");
    float *dst[LB_NFIELDS] = {};
    float *stage = (float *)c->pop[c->cur ^ 1];  // the idle population buffer stages host outputs
    for (int j = 0; j < LB_NFIELDS; ++j) {
        if (!(mask & (1u << j))) continue;
        if (!outs[j]) return fail(LB_EINVAL, "outs[" + std::to_string(j) + "] is NULL but selected");
        dst[j] = on_device ? outs[j] : stage + (long long)j * c->nn;
    }
    const StepArgs sa = state_args(c);
    FieldOut fo;
    for (int j = 0; j < LB_NFIELDS; ++j) fo.o[j] = dst[j];
    if (c->p.storage == LB_STORE_FP16)
        fields_kernel<STORE_FP16><<<grid_for(c->nn, 256), 256, 0, c->stream>>>(sa, fo, sa.gx, sa.gy, sa.gz);
    else if (c->p.storage == LB_STORE_FP16_FIT)
        fields_kernel<STORE_FP16_FIT><<<grid_for(c->nn, 256), 256, 0, c->stream>>>(sa, fo, sa.gx, sa.gy, sa.gz);
    else
        fields_kernel<STORE_FP32><<<grid_for(c->nn, 256), 256, 0, c->stream>>>(sa, fo, sa.gx, sa.gy, sa.gz);
    c->launches += 1;
    LB_CUDA(cudaGetLastError());
    if (!on_device) {
        for (int j = 0; j < LB_NFIELDS; ++j)
            if (dst[j]) LB_CUDA(cudaMemcpyAsync(outs[j], dst[j], c->nn * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
        LB_CUDA(cudaStreamSynchronize(c->stream));
    }
    return LB_OK;
}

lb_status lb_populations(lb_ctx *c, float *out, int32_t on_device) {
    if (!c || !out) return fail(LB_EINVAL, "ctx and out must not be NULL");
    if (!c->initialized) return fail(LB_ESTATE, "lb_populations before lb_init/lb_load");
    // decode one colour at a time (27 x nodes floats); host output is staged in the idle
    // population buffer, which holds at least one colour in either storage
    const StepArgs sa = state_args(c);
    float *stage = (float *)c->pop[c->cur ^ 1];
    const size_t cbytes = (size_t)27 * c->nn * sizeof(float);
    for (int k = 0; k < 2; ++k) {
        float *dst = on_device ? out + (size_t)k * 27 * c->nn : stage;
        if (c->p.storage == LB_STORE_FP16)
            canonical_kernel<STORE_FP16><<<grid_for(c->nn, 256), 256, 0, c->stream>>>(sa, k, dst);
        else if (c->p.storage == LB_STORE_FP16_FIT)
            canonical_kernel<STORE_FP16_FIT><<<grid_for(c->nn, 256), 256, 0, c->stream>>>(sa, k, dst);
        else
            canonical_kernel<STORE_FP32><<<grid_for(c->nn, 256), 256, 0, c->stream>>>(sa, k, dst);
        c->launches += 1;
        LB_CUDA(cudaGetLastError());
        if (!on_device)
            LB_CUDA(cudaMemcpyAsync(out + (size_t)k * 27 * c->nn, stage, cbytes, cudaMemcpyDeviceToHost, c->stream));
    }
    if (!on_device) LB_CUDA(cudaStreamSynchronize(c->stream));
    return LB_OK;
}

lb_status lb_history(lb_ctx *c, float *out, int32_t on_device) {
    if (!c || !out) return fail(LB_EINVAL, "ctx and out must not be NULL");
    if (!c->initialized) return fail(LB_ESTATE, "lb_history before lb_init/lb_load");
    LB_CUDA(cudaMemcpyAsync(out, c->hist[c->hcur], (size_t)54 * c->plane * sizeof(float),
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    if (!on_device) LB_CUDA(cudaStreamSynchronize(c->stream));
    return LB_OK;
}

lb_status lb_mass_noalloc(const float *pop, int64_t nodes, double *out, void *stream) {
    if (!pop || !out) return fail(LB_EINVAL, "pop and out must be device pointers, not NULL");
    if (nodes < 1 || nodes > LB_MASS_NOALLOC_MAX_NODES)
        return fail(LB_EINVAL, "lb_mass_noalloc: nodes must lie in [1, " + std::to_string(LB_MASS_NOALLOC_MAX_NODES) +
                                   "] (static scratch of " + std::to_string(LB_MASS_NOALLOC_MAX_BLOCKS) +
                                   " blocks per colour); got " + std::to_string(nodes));
    // Device address of the scratch array for the current device and context, looked up on
    // every call (in host code the array's name is only a host-side stand-in, and a cached
    // address would go stale after cudaDeviceReset or a new primary context).  The lookup
    // allocates nothing; on the first call on a device it also loads the library's device code
    // there.
    void *sym = nullptr;
    {
        cudaError_t e = cudaGetSymbolAddress(&sym, g_mass_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_mass_noalloc_scratch)");
    }
    double *scratch = (double *)sym;
    const int nblocks = (int)((nodes + LB_MASS_NOALLOC_CHUNK - 1) / LB_MASS_NOALLOC_CHUNK);
    cudaStream_t s = (cudaStream_t)stream;
    mass_partial_kernel<<<dim3(nblocks, 2), kMassThreads, 0, s>>>(pop, nodes, scratch);
    mass_final_kernel<<<1, 1024, 0, s>>>(scratch, nblocks, scratch + 2 * LB_MASS_NOALLOC_MAX_BLOCKS);
    LB_CUDA(cudaGetLastError());
    LB_CUDA(cudaMemcpyAsync(out, scratch + 2 * LB_MASS_NOALLOC_MAX_BLOCKS, 2 * sizeof(double),
                            cudaMemcpyDeviceToDevice, s));
    return LB_OK;
}

lb_status lb_mass(lb_ctx *c, double out[2]) {
    if (!c || !out) return fail(LB_EINVAL, "ctx and out must not be NULL");
    if (!c->initialized) return fail(LB_ESTATE, "lb_mass before lb_init/lb_load");
    return run_mass(c, out);
}

struct SaveHeader {
    uint64_t magic;
    int32_t nx, ny, nz, storage;
    int64_t step;
    uint64_t pop_bytes, hist_bytes;
};

// Checkpoint layout: header, the raw current population buffer (internal storage layout),
// for FP16 storage the phase entries it was encoded for, then the outflow history plane.
static size_t shift_bytes(const lb_ctx *c) { return c->p.storage == LB_STORE_FP32 ? 0 : 16 * (size_t)c->nn; }

lb_status lb_save(lb_ctx *c, void *buf, size_t *nbytes) {
    if (!c || !nbytes) return fail(LB_EINVAL, "ctx and nbytes must not be NULL");
    if (!c->initialized) return fail(LB_ESTATE, "lb_save before lb_init/lb_load");
    const size_t pb = pop_buffer_bytes(c->nn, c->p.storage), sb = shift_bytes(c);
    const size_t hb = (size_t)54 * c->plane * sizeof(float);
    const size_t total = sizeof(SaveHeader) + pb + sb + hb;
    if (!buf) {
        *nbytes = total;
        return LB_OK;
    }
    if (*nbytes < total) return fail(LB_EINVAL, "checkpoint buffer too small");
    SaveHeader h{kMagic, c->g.nx, c->g.ny, c->g.nz, c->p.storage, c->step, pb + sb, hb};
    std::memcpy(buf, &h, sizeof(h));
    char *p = (char *)buf + sizeof(h);
    LB_CUDA(cudaMemcpyAsync(p, c->pop[c->cur], pb, cudaMemcpyDeviceToHost, c->stream));
    if (sb) LB_CUDA(cudaMemcpyAsync(p + pb, c->ph4[c->cur], sb, cudaMemcpyDeviceToHost, c->stream));
    LB_CUDA(cudaMemcpyAsync(p + pb + sb, c->hist[c->hcur], hb, cudaMemcpyDeviceToHost, c->stream));
    LB_CUDA(cudaStreamSynchronize(c->stream));
    *nbytes = total;
    return LB_OK;
}

lb_status lb_load(lb_ctx *c, const void *buf, size_t nbytes) {
    if (!c || !buf) return fail(LB_EINVAL, "ctx and buf must not be NULL");
    if (nbytes < sizeof(SaveHeader)) return fail(LB_EINVAL, "checkpoint too small");
    SaveHeader h;
    std::memcpy(&h, buf, sizeof(h));
    const size_t pb = pop_buffer_bytes(c->nn, c->p.storage), sb = shift_bytes(c);
    const size_t hb = (size_t)54 * c->plane * sizeof(float);
    if (h.magic != kMagic || h.nx != c->g.nx || h.ny != c->g.ny || h.nz != c->g.nz || h.storage != c->p.storage ||
        h.pop_bytes != pb + sb || h.hist_bytes != hb || nbytes < sizeof(h) + pb + sb + hb)
        return fail(LB_EINVAL, "checkpoint does not match this context (grid, storage or size)");
    const char *p = (const char *)buf + sizeof(h);
    c->cur = 0;
    c->hcur = 0;
    LB_CUDA(cudaMemcpyAsync(c->pop[0], p, pb, cudaMemcpyHostToDevice, c->stream));
    if (sb) LB_CUDA(cudaMemcpyAsync(c->ph4[0], p + pb, sb, cudaMemcpyHostToDevice, c->stream));
    LB_CUDA(cudaMemcpyAsync(c->hist[0], p + pb + sb, hb, cudaMemcpyHostToDevice, c->stream));
    LB_CUDA(cudaStreamSynchronize(c->stream));
    c->step = h.step;
    c->initialized = true;
    c->half = false;
    return LB_OK;
}

lb_status lb_profile_enable(lb_ctx *c, int32_t capacity) {
    if (!c) return fail(LB_EINVAL, "ctx must not be NULL");
    if (capacity < 0) return fail(LB_EINVAL, "capacity must be >= 0");
    LB_CUDA(cudaStreamSynchronize(c->stream));
    free_profile(c);
    c->prof_ev.resize(4 * (size_t)capacity);
    c->prof_fused.assign((size_t)capacity, 0);
    for (auto &e : c->prof_ev) LB_CUDA(cudaEventCreate(&e));
    c->prof_cap = capacity;
    return LB_OK;
}

lb_status lb_profile_read(lb_ctx *c, double *ms, int64_t *launches, int32_t n_kinds) {
    if (!c || !ms || !launches) return fail(LB_EINVAL, "ctx, ms and launches must not be NULL");
    LB_CUDA(cudaStreamSynchronize(c->stream));
    double acc[LB_NKERNELS] = {0, 0, 0, 0};
    int64_t cnt[LB_NKERNELS] = {0, 0, 0, 0};
    const bool planes = c->g.bc_zlo != LB_BC_PERIODIC || c->g.bc_zhi != LB_BC_PERIODIC;
    for (int s = 0; s < c->prof_used; ++s) {
        cudaEvent_t *ev = &c->prof_ev[4 * (size_t)s];
        float t;
        for (int k = 0; k < 3; ++k) {
            if (k == LB_KERNEL_BOUNDARY && !planes) continue;
            if (c->prof_fused[s] && k == LB_KERNEL_COLLIDE) continue;
            const int kind = (c->prof_fused[s] && k == LB_KERNEL_GATHER) ? LB_KERNEL_STEP : k;
            LB_CUDA(cudaEventElapsedTime(&t, ev[k], ev[k + 1]));
            acc[kind] += t;
            cnt[kind] += 1;
        }
    }
    for (int k = 0; k < n_kinds && k < LB_NKERNELS; ++k) {
        ms[k] = acc[k];
        launches[k] = cnt[k];
    }
    c->prof_used = 0;
    return LB_OK;
}

int64_t lb_kernel_launches(const lb_ctx *c) { return c ? c->launches : -1; }

lb_status lb_selftest(lb_ctx *c, int32_t which, int32_t *result, double *ms) {
    if (!c || !result || !ms) return fail(LB_EINVAL, "ctx, result and ms must not be NULL");
    if (which != LB_SELFTEST_FUSED_WAIT) return fail(LB_EINVAL, "unknown self-test");
    if (c->half) return fail(LB_ESTATE, "lb_selftest inside a split step");
    // the fused kernel's wait on plane 0 with a target no counter reaches; the scratch of the
    // mass reduction takes the waited time
    FusedCtl f{};
    f.done = c->fdone;
    f.err = c->ferr;
    f.target = ~0ull;
    unsigned long long *ns = reinterpret_cast<unsigned long long *>(c->partial);
    LB_CUDA(launch_fused_wait_probe(f, ns, c->stream));
    c->launches += 1;
    unsigned long long waited = 0;
    int err = 0;
    LB_CUDA(cudaMemcpyAsync(&waited, ns, sizeof(waited), cudaMemcpyDeviceToHost, c->stream));
    LB_CUDA(cudaMemcpyAsync(&err, c->ferr, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    LB_CUDA(cudaStreamSynchronize(c->stream));
    LB_CUDA(cudaMemsetAsync(c->ferr, 0, sizeof(int), c->stream));
    LB_CUDA(cudaStreamSynchronize(c->stream));
    *result = err ? LB_ETIMEOUT : LB_OK;
    *ms = (double)waited * 1e-6;
    return LB_OK;
}

lb_status lb_adjoint(lb_ctx *c, int32_t objective, int64_t T, const double *obj_args, double *grad_out,
                     int32_t n_grad) {
    if (!c || !obj_args || !grad_out) return fail(LB_EINVAL, "ctx, obj_args and grad_out must not be NULL");
    if (!c->initialized) return fail(LB_ESTATE, "lb_adjoint before lb_init/lb_load");
    if (c->half) return fail(LB_ESTATE, "lb_adjoint inside a split step");
    if (c->p.storage != LB_STORE_FP32) return fail(LB_EINVAL, "lb_adjoint needs FP32 population storage");
    if (c->p.s3 != 1.0 || c->p.s4 != 1.0 || c->p.s5 != 1.0 || c->p.s6 != 1.0)
        return fail(LB_EINVAL, "lb_adjoint needs the paper's rates s3 = s4 = s5 = s6 = 1");
    if (T < 1) return fail(LB_EINVAL, "T must be >= 1");
    if (n_grad < LB_ADJ_NOUT) return fail(LB_EINVAL, "grad_out must hold LB_ADJ_NOUT doubles");
    for (int j = 0; j < LB_ADJ_NARGS; ++j)
        if (!std::isfinite(obj_args[j])) return fail(LB_EINVAL, "obj_args must be finite");
    if (objective == LB_OBJ_INTERFACE_AREA) {
        if (!(obj_args[0] > 0)) return fail(LB_EINVAL, "interface area needs eps = obj_args[0] > 0");
    } else if (objective == LB_OBJ_PENETRATION) {
        if (!(obj_args[0] > 0)) return fail(LB_EINVAL, "penetration length needs delta = obj_args[0] > 0");
    } else {
        return fail(LB_EINVAL, "unknown objective");
    }
    if (obj_args[2] < 0) return fail(LB_EINVAL, "checkpoint interval obj_args[2] must be >= 0");
    long long k = obj_args[2] >= 1 ? (long long)obj_args[2] : (long long)std::ceil(std::sqrt((double)T));
    k = std::max(1ll, std::min<long long>(k, T));
    const long long nseg = (T + k - 1) / k;

    // workspace: checkpoints every k steps; two sets of per-step records (one segment is
    // recomputed into one set while the reverse sweep steps back through the other); the
    // adjoint state
    const size_t NN = (size_t)c->nn, P = (size_t)c->plane;
    const size_t pb = 27 * NN * sizeof(float2), hb = 54 * P * sizeof(float), nb2 = NN * sizeof(float2);
    StepArgs a0 = make_args(c);
    const long long nblk_coll = adj_collide_blocks(a0), nblk_inlet = adj_boundary_blocks(a0);
    // per recorded step: the collision inputs (the moment pass's 48 B and the 24 B of gradients
    // a node), f(N-1) and hist(n+1) of the outflow plane; the recomputed populations
    // themselves only in two alternating buffers
    const size_t rmom = k * 3 * NN * sizeof(float4), rg4 = k * NN * sizeof(float4), rg2 = k * nb2, rfm = k * hb,
                 rhist = (k + 1) * hb;
    const size_t parts[] = {nseg * pb, nseg * hb, 2 * pb, rmom, rg4, rg2, rfm, rhist, rmom, rg4, rg2, rfm, rhist,
                            pb, pb, nb2, nb2, NN * sizeof(float4), nb2, hb, 9 * P * sizeof(float), hb, hb,
                            nblk_coll * 3 * sizeof(double), nblk_inlet * 17 * sizeof(double),
                            nblk_coll * sizeof(double), 32 * sizeof(double), nb2};
    constexpr int kParts = (int)(sizeof(parts) / sizeof(parts[0]));
    size_t need = 0;
    for (size_t v : parts) need += align_up(v);
    if (need > c->adj.bytes) {
        if (c->adj.base) cudaFree(c->adj.base);
        c->adj.base = nullptr;
        c->adj.bytes = 0;
        c->adj.valid = false;
        if (cudaMalloc(&c->adj.base, need) != cudaSuccess) {
            cudaGetLastError();
            return fail(LB_ENOMEM, "cannot allocate the adjoint workspace (" + std::to_string(need >> 20) + " MiB)");
        }
        c->adj.bytes = need;
    }
    {
        char *p = (char *)c->adj.base;
        size_t j = 0;
        auto take = [&](void *&dst) { dst = p; p += align_up(parts[j++]); };
        void *v[kParts];
        for (int q = 0; q < kParts; ++q) take(v[q]);
        auto &w = c->adj;
        w.ckpt_pop = (float2 *)v[0]; w.ckpt_hist = (float *)v[1]; w.seg_pop = (float2 *)v[2];
        for (int r = 0; r < 2; ++r) {
            w.seg_mom[r] = (float4 *)v[3 + 5 * r]; w.seg_g4[r] = (float4 *)v[4 + 5 * r];
            w.seg_g2[r] = (float2 *)v[5 + 5 * r]; w.seg_fm[r] = (float *)v[6 + 5 * r];
            w.seg_hist[r] = (float *)v[7 + 5 * r];
        }
        w.lp[0] = (float2 *)v[13]; w.lp[1] = (float2 *)v[14]; w.lr[0] = (float2 *)v[15];
        w.lr[1] = (float2 *)v[16]; w.lga = (float4 *)v[17]; w.lgb = (float2 *)v[18]; w.lc = (float *)v[19];
        w.li = (float *)v[20]; w.lh[0] = (float *)v[21]; w.lh[1] = (float *)v[22]; w.acc_coll = (double *)v[23];
        w.acc_inlet = (double *)v[24]; w.acc_obj = (double *)v[25]; w.out = (double *)v[26];
        w.objph = (float2 *)v[27];
        w.nblk_coll = nblk_coll;
        w.nblk_inlet = nblk_inlet;
    }
    auto &w = c->adj;
    w.valid = false;
    if (!w.s2) {
        LB_CUDA(cudaStreamCreateWithFlags(&w.s2, cudaStreamNonBlocking));
        LB_CUDA(cudaEventCreateWithFlags(&w.ev_fwd, cudaEventDisableTiming));
        for (int r = 0; r < 2; ++r) {
            LB_CUDA(cudaEventCreateWithFlags(&w.ev_rec[r], cudaEventDisableTiming));
            LB_CUDA(cudaEventCreateWithFlags(&w.ev_rev[r], cudaEventDisableTiming));
        }
    }
    const bool conv = c->g.bc_zhi == LB_BC_CONVECTIVE;
    cudaStream_t st = c->stream, s2 = w.s2;
    LB_CUDA(cudaMemsetAsync(w.acc_coll, 0, nblk_coll * 3 * sizeof(double), st));
    LB_CUDA(cudaMemsetAsync(w.acc_inlet, 0, nblk_inlet * 17 * sizeof(double), st));
    LB_CUDA(cudaMemsetAsync(w.acc_obj, 0, nblk_coll * sizeof(double), st));
    LB_CUDA(cudaMemsetAsync(w.out, 0, 32 * sizeof(double), st));
    LB_CUDA(cudaMemsetAsync(w.lh[0], 0, hb, st));
    LB_CUDA(cudaMemsetAsync(w.lc, 0, hb, st));
    LB_CUDA(cudaMemsetAsync(w.li, 0, 9 * P * sizeof(float), st));

    // what the reverse needs of step t of a segment (record set r = segment index & 1): the
    // collision inputs, f(N-1) and the outflow history before and after the step
    auto record = [&](StepArgs &a, long long t, int r) {
        a.hist_in = w.seg_hist[r] + t * 54 * P;
        a.hist_out = w.seg_hist[r] + (t + 1) * 54 * P;
        a.mom = w.seg_mom[r] + t * 3 * NN;
        a.grad4 = w.seg_g4[r] + t * NN;
        a.grad2 = w.seg_g2[r] + t * NN;
        a.fm_out = conv ? w.seg_fm[r] + t * 54 * P : nullptr;
    };
    // forward pass with a checkpoint at the start of every segment; the last segment records
    // as it goes, so the reverse sweep needs no recompute for it
    const int64_t step0 = c->step;
    for (long long sg = 0; sg < nseg; ++sg) {
        const long long len = std::min<long long>(k, T - sg * k);
        const bool last = sg == nseg - 1;
        const int r = (int)(sg & 1);
        if (!last) {  // the recorded last segment is never recomputed
            LB_CUDA(cudaMemcpyAsync(w.ckpt_pop + sg * 27 * NN, c->pop[c->cur], pb, cudaMemcpyDeviceToDevice, st));
            if (conv)
                LB_CUDA(cudaMemcpyAsync(w.ckpt_hist + sg * 54 * P, c->hist[c->hcur], hb, cudaMemcpyDeviceToDevice, st));
        }
        if (last) LB_CUDA(cudaMemcpyAsync(w.seg_hist[r], c->hist[c->hcur], hb, cudaMemcpyDeviceToDevice, st));
        for (long long t = 0; t < len; ++t) {
            StepArgs a = make_args(c);
            if (last) record(a, t, r);
            cudaError_t e = launch_step(a, LB_STORE_FP32, st, nullptr, &c->launches);
            if (e != cudaSuccess) return cuda_fail(e, "launch_step");
            c->cur ^= 1;
            if (conv && !last) c->hcur ^= 1;
            c->step += 1;
        }
        if (last && conv)
            LB_CUDA(cudaMemcpyAsync(c->hist[c->hcur], w.seg_hist[r] + len * 54 * P, hb, cudaMemcpyDeviceToDevice, st));
    }

    // objective of S(T) and its adjoint
    AdjArgs g{};
    g.lga = w.lga; g.lgb = w.lgb; g.lc = w.lc; g.li = w.li;
    g.acc_coll = w.acc_coll; g.acc_inlet = w.acc_inlet;
    int cl = 0, ch = 0;
    {
        AdjArgs go = g;
        go.lp_out = w.lp[cl];
        go.lr_out = w.lr[cl];
        cudaError_t e = launch_objective(state_args(c), go, objective, obj_args, w.objph, w.lr[cl ^ 1], w.acc_obj,
                                         w.out + 24, st, &c->launches);
        if (e != cudaSuccess) return cuda_fail(e, "launch_objective");
    }

    // reverse sweep.  Segment sg is recomputed from its checkpoint on the second stream into
    // record set sg & 1 while the context's stream steps back through segment sg + 1 (set
    // (sg + 1) & 1); the recompute of a segment waits for the reverse that last used its set,
    // the reverse of a segment for its recompute.  The recompute alone uses the population
    // buffers seg_pop and the context's phase field, moments and boundary planes (the reverse
    // kernels read none of them).
    auto seg_args = [&](long long t, int64_t step, int r) {
        StepArgs a = make_args(c);
        a.pin = w.seg_pop + (t & 1) * 27 * NN;
        a.pout = w.seg_pop + ((t + 1) & 1) * 27 * NN;
        record(a, t, r);
        a.step = step;
        return a;
    };
    LB_CUDA(cudaEventRecord(w.ev_fwd, st));
    LB_CUDA(cudaStreamWaitEvent(s2, w.ev_fwd, 0));
    auto recompute = [&](long long sg) -> lb_status {
        const int r = (int)(sg & 1);
        const long long n0 = sg * k, len = std::min<long long>(k, T - n0);
        LB_CUDA(cudaMemcpyAsync(w.seg_pop, w.ckpt_pop + sg * 27 * NN, pb, cudaMemcpyDeviceToDevice, s2));
        if (conv)
            LB_CUDA(cudaMemcpyAsync(w.seg_hist[r], w.ckpt_hist + sg * 54 * P, hb, cudaMemcpyDeviceToDevice, s2));
        for (long long t = 0; t < len; ++t) {
            cudaError_t e = launch_step(seg_args(t, step0 + n0 + t, r), LB_STORE_FP32, s2, nullptr, &c->launches);
            if (e != cudaSuccess) return cuda_fail(e, "launch_step (recompute)");
        }
        LB_CUDA(cudaEventRecord(w.ev_rec[r], s2));
        return LB_OK;
    };
    if (nseg >= 2) {
        lb_status rs = recompute(nseg - 2);
        if (rs != LB_OK) return rs;
    }
    for (long long sg = nseg - 1; sg >= 0; --sg) {
        const int r = (int)(sg & 1);
        const long long n0 = sg * k, len = std::min<long long>(k, T - n0);
        if (sg != nseg - 1) LB_CUDA(cudaStreamWaitEvent(st, w.ev_rec[r], 0));
        for (long long t = len - 1; t >= 0; --t) {
            AdjArgs gs = g;
            gs.mom = w.seg_mom[r] + t * 3 * NN;
            gs.grad4 = w.seg_g4[r] + t * NN;
            gs.grad2 = w.seg_g2[r] + t * NN;
            gs.fm = w.seg_fm[r] + t * 54 * P;
            gs.lp_in = w.lp[cl]; gs.lr_in = w.lr[cl];
            gs.lp_out = w.lp[cl ^ 1]; gs.lr_out = w.lr[cl ^ 1];
            gs.lh_in = w.lh[ch]; gs.lh_out = w.lh[ch ^ 1];
            cudaError_t e = launch_adjoint_step(seg_args(t, step0 + n0 + t, r), gs, st, &c->launches);
            if (e != cudaSuccess) return cuda_fail(e, "launch_adjoint_step");
            cl ^= 1;
            if (conv) ch ^= 1;
        }
        LB_CUDA(cudaEventRecord(w.ev_rev[r], st));
        if (sg >= 2) {  // segment sg - 2 reuses this set
            LB_CUDA(cudaStreamWaitEvent(s2, w.ev_rev[r], 0));
            lb_status rs = recompute(sg - 2);
            if (rs != LB_OK) return rs;
        }
    }
    {
        cudaError_t e = launch_adjoint_reduce(g, nblk_coll, nblk_inlet, w.out, st, &c->launches);
        if (e != cudaSuccess) return cuda_fail(e, "launch_adjoint_reduce");
    }
    double host[32];
    LB_CUDA(cudaMemcpyAsync(host, w.out, sizeof(host), cudaMemcpyDeviceToHost, st));
    LB_CUDA(cudaStreamSynchronize(st));
    grad_out[0] = host[24];
    for (int j = 1; j < LB_ADJ_NOUT; ++j) grad_out[j] = host[j];
    w.cl = cl;
    w.valid = true;
    return LB_OK;
}

lb_status lb_fragments(lb_ctx *c, int32_t connectivity, int32_t exclude_inlet, int64_t *roots, int64_t *volumes,
                       double *diameters, int64_t cap, lb_fragment_stats *stats) {
    if (!c || !stats) return fail(LB_EINVAL, "ctx and stats must not be NULL");
    if (!c->initialized) return fail(LB_ESTATE, "lb_fragments before lb_init/lb_load");
    if (connectivity != 6 && connectivity != 26) return fail(LB_EINVAL, "connectivity must be 6 or 26");
    if (cap < 0) return fail(LB_EINVAL, "cap must be >= 0");
    const size_t NN = (size_t)c->nn;
    const long long nblk = ((long long)NN + 1023) / 1024;
    // scratch: label, count (int32), touch (u8), block counts, block offsets, error flag
    const size_t parts[] = {NN * 4, NN * 4, NN, (size_t)nblk * 4, (size_t)(nblk + 1) * 8, 16};
    size_t need = 0;
    for (size_t v : parts) need += align_up(v);
    char *base = nullptr;
    if (cudaMalloc(&base, need) != cudaSuccess) {
        cudaGetLastError();
        return fail(LB_ENOMEM, "cannot allocate fragment scratch");
    }
    struct Free { char *p; ~Free() { cudaFree(p); } } guard{base};
    char *q = base;
    int *label = (int *)q; q += align_up(parts[0]);
    int *count = (int *)q; q += align_up(parts[1]);
    uint8_t *touch = (uint8_t *)q; q += align_up(parts[2]);
    int *bc = (int *)q; q += align_up(parts[3]);
    long long *boff = (long long *)q; q += align_up(parts[4]);
    int *err = (int *)q;
    cudaStream_t st = c->stream;
    LB_CUDA(cudaMemsetAsync(count, 0, NN * 4, st));
    LB_CUDA(cudaMemsetAsync(touch, 0, NN, st));
    LB_CUDA(cudaMemsetAsync(err, 0, 4, st));
    const StepArgs sa = state_args(c);
    cudaError_t e = launch_fragments_label(sa, c->p.storage, connectivity, label, count, touch, bc, boff, err, st,
                                           &c->launches);
    if (e != cudaSuccess) return cuda_fail(e, "launch_fragments_label");
    long long nroots = 0;
    int herr = 0;
    LB_CUDA(cudaMemcpyAsync(&nroots, boff + nblk, sizeof(nroots), cudaMemcpyDeviceToHost, st));
    LB_CUDA(cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, st));
    LB_CUDA(cudaStreamSynchronize(st));
    if (herr) return fail(LB_ECUDA, "fragment labelling exceeded its iteration bound");
    std::vector<long long> hroot((size_t)nroots), hvol((size_t)nroots);
    std::vector<uint8_t> htouch((size_t)nroots);
    if (nroots > 0) {
        char *ob = nullptr;
        if (cudaMalloc(&ob, (size_t)nroots * 17 + 64) != cudaSuccess) {
            cudaGetLastError();
            return fail(LB_ENOMEM, "cannot allocate the fragment list");
        }
        Free og{ob};
        long long *o_root = (long long *)ob, *o_vol = o_root + nroots;
        uint8_t *o_touch = (uint8_t *)(o_vol + nroots);
        e = launch_fragments_write(sa, connectivity, label, count, touch, boff, o_root, o_vol, o_touch, st,
                                   &c->launches);
        if (e != cudaSuccess) return cuda_fail(e, "launch_fragments_write");
        LB_CUDA(cudaMemcpyAsync(hroot.data(), o_root, (size_t)nroots * 8, cudaMemcpyDeviceToHost, st));
        LB_CUDA(cudaMemcpyAsync(hvol.data(), o_vol, (size_t)nroots * 8, cudaMemcpyDeviceToHost, st));
        LB_CUDA(cudaMemcpyAsync(htouch.data(), o_touch, (size_t)nroots, cudaMemcpyDeviceToHost, st));
        LB_CUDA(cudaStreamSynchronize(st));
    }
    // kept fragments, diameters and the mass-median diameter (sorted by volume, ties by root)
    const bool drop_column = exclude_inlet && c->g.bc_zlo == LB_BC_INLET;
    std::vector<long long> kr, kv;
    long long column = 0, total = 0;
    for (long long k = 0; k < nroots; ++k) {
        if (drop_column && htouch[(size_t)k]) {
            column += hvol[(size_t)k];
            continue;
        }
        kr.push_back(hroot[(size_t)k]);
        kv.push_back(hvol[(size_t)k]);
        total += hvol[(size_t)k];
    }
    double dm = 0.0;
    if (!kv.empty()) {
        std::vector<size_t> order(kv.size());
        for (size_t k = 0; k < order.size(); ++k) order[k] = k;
        std::stable_sort(order.begin(), order.end(), [&](size_t i, size_t j) { return kv[i] < kv[j]; });
        long long cum = 0;
        for (size_t k : order) {
            cum += kv[k];
            if (2 * cum >= total) {
                dm = std::cbrt(6.0 * (double)kv[k] / 3.14159265358979323846);
                break;
            }
        }
    }
    for (long long k = 0; k < (long long)kr.size() && k < cap; ++k) {
        if (roots) roots[k] = kr[(size_t)k];
        if (volumes) volumes[k] = kv[(size_t)k];
        if (diameters) diameters[k] = std::cbrt(6.0 * (double)kv[(size_t)k] / 3.14159265358979323846);
    }
    stats->n_fragments = (int64_t)kr.size();
    stats->column_volume = column;
    stats->total_volume = total;
    stats->mass_median_diameter = dm;
    return LB_OK;
}

lb_status lb_adjoint_state(lb_ctx *c, float *out, int32_t on_device) {
    if (!c || !out) return fail(LB_EINVAL, "ctx and out must not be NULL");
    if (!c->adj.valid) return fail(LB_ESTATE, "lb_adjoint_state before a successful lb_adjoint");
    auto &w = c->adj;
    AdjArgs g{};
    g.lp_in = w.lp[w.cl];
    g.lr_in = w.lr[w.cl];
    const size_t bytes = 54 * (size_t)c->nn * sizeof(float);
    float *dst = on_device ? out : (float *)w.lp[w.cl ^ 1];
    cudaError_t e = launch_adjoint_state(make_args(c), g, dst, c->stream, &c->launches);
    if (e != cudaSuccess) return cuda_fail(e, "launch_adjoint_state");
    if (!on_device) LB_CUDA(cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, c->stream));
    LB_CUDA(cudaStreamSynchronize(c->stream));
    return LB_OK;
}

}  // extern "C"
