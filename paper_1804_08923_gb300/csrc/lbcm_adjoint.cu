// lbcm_adjoint.cu -- discrete adjoint (reverse mode) of the FP32 step with the paper's rates
// s3 = s4 = s5 = s6 = 1 (arXiv:1804.08923, Section II; boundaries of Section IV.A).
//
// The step S(n) -> S(n+1) is
//   stream (pull, inlet / mirror / convective outflow)  f = P(S(n), hist(n))
//   densities and isotropic gradients                   rho_k = sum_i f_i^k, grad phi, grad rho
//   per-node collision, perturbation, recolouring        S(n+1) = C(f, grad phi, grad rho)
// and its transpose, given lambda = dJ/dS(n+1), runs in three launches:
//   adj_collide_kernel   per node: recomputes the node's forward quantities from S(n) and the
//                        saved phase field, applies (dC/df)^T, (dC/dgrad)^T and accumulates
//                        dJ/d(sigma, nu_r, nu_b); pushes lambda_f to the slots of S(n) its pulls
//                        read (the transposed streaming), writes lambda of the two gradients.
//   adj_stencil_kernel   per node: transposes the gradient stencil (with the ghost rules) into
//                        lambda_rho_k, the adjoint of the node's colour densities.  It is added
//                        to every population the node pulled, i.e. "deferred" to the reader in
//                        the next reverse step instead of another full pass.
//   adj_boundary_kernel  per (x, y) column: inlet-disc gradients w.r.t. u_in and the 16 profile
//                        coefficients, and the transpose of the convective outflow
//                        f(N) = [hist + lambda f(N-1)] / (1 + lambda), lambda = clamp(u_z(N-1)).
// The adjoint state between steps is (Lp, Lr, Lh): lambda_S(n)(x, k, i) = Lp(x, k, i) +
// Lr^k(reader of slot (x, i)), and Lh = dJ/dhist(n).  Parameter gradients are summed per
// block in FP64 into one accumulator slot per block (deterministic, no atomics).
#include "lbcm_device.cuh"
#include "lbcm_internal.h"
#include "lbcm_node.cuh"

#include <algorithm>

namespace lbcm {

// Adds the block sums of v[0..NV) to acc[blk * NV + k] (FP64).  The sum over the block's
// threads is FP32 (shuffles, then one warp over the warp sums); only the block total is
// converted and accumulated in FP64, since FP64 throughput is a small fraction of FP32 here.
// Every thread of the block must call it (no early return before).
template <int NV>
__device__ __forceinline__ void block_accumulate(const float (&v)[NV], double *acc, long long blk) {
    __shared__ float sh[NV][32];
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int lane = tid & 31, warp = tid >> 5, nwarp = (nthr + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        float d = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
        if (lane == 0) sh[k][warp] = d;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            float d = lane < nwarp ? sh[k][lane] : 0.0f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
            if (lane == 0) acc[blk * NV + k] += (double)d;
        }
    }
}

__device__ __forceinline__ long long block_id() {
    return blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
}

// Whether a pull of step n+1 reads slot (node at height z, direction i): the inlet disc and the
// convective plane read nothing.
__device__ __forceinline__ bool slot_read(const StepArgs &a, int i, int z, bool own_in_disc) {
    if (a.bc_zlo == BC_PERIODIC) return true;
    const int zr = z + cz(i);
    if (a.bc_zhi == BC_CONVECTIVE && zr >= a.nz - 1) return false;
    return !(zr < 0 && own_in_disc);
}

// lambda_S(n+1) of slot (node nb.n, direction i): the pushed part plus the deferred density
// adjoint of the node that reads the slot in step n+1, if a pull reads it.
__device__ __forceinline__ float2 adj_slot(const StepArgs &a, const AdjArgs &g, const Nbr &nb, int i, int z,
                                           bool own_in_disc) {
    float2 v = __ldg(g.lp_in + (size_t)i * a.NN + nb.n);
    if (slot_read(a, i, z, own_in_disc)) {
        const float2 r = __ldg(g.lr_in + nb.nbr(i));
        v.x += r.x;
        v.y += r.y;
    }
    return v;
}

// 8-byte asynchronous global -> shared copy (no register holds the value in flight).
__device__ __forceinline__ void cp_async8(unsigned smem, const void *gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// 1-D transpose of the inverse sweep: M_a = sum_c v_c G_a[c](u) for a = 0, 1, 2.
__device__ __forceinline__ void sweep_inv_T(float &a0, float &a1, float &a2, const InvAxis &A) {
    const float v0 = a0, v1 = a1, v2 = a2;
    a0 = fmaf(A.g0[0], v0, fmaf(A.g0[1], v1, A.g0[2] * v2));
    a1 = fmaf(A.g1[0], v0, fmaf(A.g1[1], v1, A.g1[2] * v2));
    a2 = fmaf(0.5f, v0 + v2, -v1);
}

// Weighted raw moments m_pqr = sum_i v_i w_i cx^p cy^q cz^r (p, q, r <= 2) of 27 values in the
// tensor layout [cx+1][cy+1][cz+1], by 1-D sweeps: D3Q27's w_i is the product of the 1-D weights
// (1/6, 2/3, 1/6).  Only the moments of total order <= 3 are kept (c^3 = c on the lattice).
struct RawMom {
    float m000, m100, m010, m001, m200, m020, m002, m110, m101, m011, m210, m201, m120, m021, m102, m012, m111;
};
__device__ __forceinline__ void wsweep(float &v0, float &v1, float &v2) {
    const float s = (v2 + v0) * (1.0f / 6.0f), d = (v2 - v0) * (1.0f / 6.0f);
    v0 = fmaf(2.0f / 3.0f, v1, s);
    v1 = d;
    v2 = s;
}
__device__ __forceinline__ void raw_moments(float (&t)[27], RawMom &M) {
#pragma unroll
    for (int q = 0; q < 9; ++q) wsweep(t[q], t[9 + q], t[18 + q]);
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int c = 0; c < 3; ++c) wsweep(t[p * 9 + c], t[p * 9 + 3 + c], t[p * 9 + 6 + c]);
#pragma unroll
    for (int p = 0; p < 9; ++p) wsweep(t[p * 3], t[p * 3 + 1], t[p * 3 + 2]);
#define T_(p, q, r) t[(p) * 9 + (q) * 3 + (r)]
    M = RawMom{T_(0, 0, 0), T_(1, 0, 0), T_(0, 1, 0), T_(0, 0, 1), T_(2, 0, 0), T_(0, 2, 0), T_(0, 0, 2), T_(1, 1, 0),
               T_(1, 0, 1), T_(0, 1, 1), T_(2, 1, 0), T_(2, 0, 1), T_(1, 2, 0), T_(0, 2, 1), T_(1, 0, 2), T_(0, 1, 2),
               T_(1, 1, 1)};
#undef T_
}
// M2 v (the second-moment tensor applied to a vector) and v.M2.w
__device__ __forceinline__ void m2v(const RawMom &M, float vx, float vy, float vz, float &ox, float &oy, float &oz) {
    ox = M.m200 * vx + M.m110 * vy + M.m101 * vz;
    oy = M.m110 * vx + M.m020 * vy + M.m011 * vz;
    oz = M.m101 * vx + M.m011 * vy + M.m002 * vz;
}
// A3(., u, u)_a = sum_i v_i w_i c_a (c.u)^2
__device__ __forceinline__ void m3uu(const RawMom &M, float ux, float uy, float uz, float &ox, float &oy, float &oz) {
    const float xx = ux * ux, yy = uy * uy, zz = uz * uz, xy = 2.0f * ux * uy, xz = 2.0f * ux * uz, yz = 2.0f * uy * uz;
    ox = M.m100 * xx + M.m120 * yy + M.m102 * zz + M.m210 * xy + M.m201 * xz + M.m111 * yz;
    oy = M.m210 * xx + M.m010 * yy + M.m012 * zz + M.m120 * xy + M.m111 * xz + M.m021 * yz;
    oz = M.m201 * xx + M.m021 * yy + M.m001 * zz + M.m111 * xy + M.m102 * xz + M.m012 * yz;
}

// Starts the copies of lambda_S(n+1) of node nb.n into shared memory: the pushed part of each
// slot, and the deferred density adjoint of the node that reads the slot in step n+1 where a
// pull reads it (else zero).  kEdge = false: the caller knows that 0 < z < N - 1, where every
// slot is read.
template <bool kEdge>
__device__ __forceinline__ void adj_fetch(const StepArgs &a, const AdjArgs &g, const Nbr &nb, int z, float2 *L_s,
                                          float2 *R_s) {
    const bool own_in_disc = kEdge && a.bc_zlo == BC_INLET && z == 0 && a.disc[nb.pxy];
    const unsigned sL = (unsigned)__cvta_generic_to_shared(L_s), sR = (unsigned)__cvta_generic_to_shared(R_s);
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        cp_async8(sL + cell(i) * 128 * 8, g.lp_in + (size_t)i * a.NN + nb.n);
        if (!kEdge || slot_read(a, i, z, own_in_disc))
            cp_async8(sR + cell(i) * 128 * 8, g.lr_in + nb.nbr(i));
        else
            R_s[cell(i) * 128] = make_float2(0.0f, 0.0f);
    }
    cp_async_commit();
}

// The adjoints of the 54 gathered populations of a node, from the adjoints of its momentum,
// raw second moment and colour densities.
struct AdjPush {
    float ljx, ljy, ljz, lQxx, lQyy, lQzz, lQxy, lQxz, lQyz, lrr, lrb;
};

// Pushes lambda_f_i of node nb.n to the slot its pull read: the transposed streaming, with the
// mirror, the inlet disc and the convective outflow on the boundary planes.  kEdge = false:
// the caller knows that 0 < z < N, and the boundary-plane tests of every direction drop out.
template <bool W, bool kEdge>
__device__ __forceinline__ void adj_push(const StepArgs &a, const AdjArgs &g, const Nbr &nb, int z, const AdjPush &q) {
    const int N = a.nz - 1;
    const bool pz = a.bc_zlo == BC_PERIODIC;
    const bool conv_top = kEdge && !pz && z == N && a.bc_zhi == BC_CONVECTIVE;
    const bool bot = kEdge && !pz && z == 0;
    const bool slip_top = kEdge && !pz && z == N && a.bc_zhi == BC_FREESLIP;
    const size_t P = (size_t)a.plane;
#define PULLED(i) (W ? nb.pulled(i) : (i))
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        const float c0 = (float)cx(i), c1 = (float)cy(i), c2 = (float)cz(i);
        float lf = c0 * q.ljx + c1 * q.ljy + c2 * q.ljz;
        lf += c0 * c0 * q.lQxx + c1 * c1 * q.lQyy + c2 * c2 * q.lQzz + c0 * c1 * q.lQxy + c0 * c2 * q.lQxz +
              c1 * c2 * q.lQyz;
        const float2 o = make_float2(lf + q.lrr, lf + q.lrb);
        if (conv_top) {
            // f(N) comes from the outflow rule: its adjoint goes to the boundary kernel; the
            // slots the plain pulls would have read are read by nobody
            g.lc[(size_t)i * P + nb.pxy] = o.x;
            g.lc[(size_t)(27 + i) * P + nb.pxy] = o.y;
            if (cz(i) >= 0) g.lp_out[(size_t)PULLED(i) * a.NN + nb.src(i)] = make_float2(0.0f, 0.0f);
            if (cz(i) == 1) g.lp_out[(size_t)i * a.NN + nb.n] = make_float2(0.0f, 0.0f);
        } else if (bot && cz(i) == 1) {
            const int xs = nb.xo[cx(i) + 1], ys = nb.yo[cy(i) + 1];  // source column (offsets, reflected)
            const size_t slot = (size_t)mirror_z(PULLED(i)) * a.NN + ys + xs;
            if (a.bc_zlo == BC_INLET && a.disc[ys + xs]) {
                g.li[(size_t)zrank(i) * P + nb.pxy] = o.x;
                g.lp_out[slot] = make_float2(0.0f, 0.0f);
            } else {
                g.lp_out[slot] = o;
            }
        } else if (slip_top && cz(i) == -1) {
            const int xs = nb.xo[cx(i) + 1], ys = nb.yo[cy(i) + 1];
            g.lp_out[(size_t)mirror_z(PULLED(i)) * a.NN + (size_t)N * P + ys + xs] = o;
        } else {
            g.lp_out[(size_t)PULLED(i) * a.NN + nb.src(i)] = o;
        }
    }
#undef PULLED
}

// ---------------------------------------------------------------- reverse collision
// Every per-direction sum of the reverse pass is linear in a_i = (rho_r lS^r_i + rho_b lS^b_i)/rho
// or b_i = lS^r_i - lS^b_i with coefficients that are polynomials in c_i times shell constants
// proportional to w_i (varphi_i(alpha) = 27/19 (1 - alpha) w_i, the Phi coefficient 9 w_i and
// B_i = w_i for i >= 1), so it is a combination of the weighted raw moments of a and b up to
// third order.  Only the recolouring's 1/|c_i| is not separable and is summed directly.
template <bool kForce, bool W>
__device__ __forceinline__ void adj_collide_node(const StepArgs &a, const AdjArgs &g, int x, int y, int z,
                                                 float (&part)[3], float2 *L_s, float2 *R_s) {
    const Nbr nb(a, x, y, z);
    const int N = a.nz - 1;

    // lambda of S(n+1) for the 27 directions: the pushed and the deferred parts are copied
    // asynchronously into this thread's two columns of shared memory (tensor layout), and the
    // node's recorded forward quantities are loaded and used while they are in flight
    if (z == 0 || z >= N - 1)
        adj_fetch<true>(a, g, nb, z, L_s, R_s);
    else
        adj_fetch<false>(a, g, nb, z, L_s, R_s);

    // ---- the forward step's collision inputs of this node (recorded in the recompute)
    const size_t NN = (size_t)a.NN;
    const Moments mo = load_moments(g.mom, NN, nb.n);
    const float4 r3 = __ldg(g.grad4 + nb.n);
    const float2 r4 = __ldg(g.grad2 + nb.n);
    const float gpx = r3.x, gpy = r3.y, gpz = r3.z, grx = r3.w, gry = r4.x, grz = r4.y;
    const float rr = mo.rho_r, rb = mo.rho_b;
    const float rho = rr + rb, inv_rho = 1.0f / rho;
    float Fx = 0.0f, Fy = 0.0f, Fz = 0.0f;
    if (kForce) {
        const float fo = rho - a.rho_b0;
        Fx = fo * a.gx; Fy = fo * a.gy; Fz = fo * a.gz;
    }
    const float ux = fmaf(0.5f, Fx, mo.jx) * inv_rho, uy = fmaf(0.5f, Fy, mo.jy) * inv_rho,
                uz = fmaf(0.5f, Fz, mo.jz) * inv_rho;
    const float phi = order_parameter(rr, rb, a.inv_rho_r0, a.inv_rho_b0);
    const float hp = 0.5f * (1.0f + phi), hm = 0.5f * (1.0f - phi);
    const float oma = one_minus_alpha_bar(a.alpha_mix, rr, rb, inv_rho, hp, hm, a.oma_r, a.oma_b), alpha = 1.0f - oma;
    const float nu = 1.0f / (hp * a.inv_nu_r + hm * a.inv_nu_b);
    const float tau = 3.0f * nu + 0.5f, s2nu = 1.0f / tau;
    const float Acoef = 2.25f * a.sigma / tau;
    const float usq = ux * ux + uy * uy + uz * uz;
    const float ugr = ux * grx + uy * gry + uz * grz;
    const float uF = ux * Fx + uy * Fy + uz * Fz;
    const float cs2 = oma * (9.0f / 19.0f);
    // Q: second central moment of f - f^e + F'/2 (Pi(f^e), Pi(F') in closed form)
    float Qxx = mo.pxx - (rho * cs2 + rho * ux * ux + nu * (2.0f * ux * grx + ugr));
    float Qyy = mo.pyy - (rho * cs2 + rho * uy * uy + nu * (2.0f * uy * gry + ugr));
    float Qzz = mo.pzz - (rho * cs2 + rho * uz * uz + nu * (2.0f * uz * grz + ugr));
    float Qxy = mo.pxy - (rho * ux * uy + nu * (ux * gry + uy * grx));
    float Qxz = mo.pxz - (rho * ux * uz + nu * (ux * grz + uz * grx));
    float Qyz = mo.pyz - (rho * uy * uz + nu * (uy * grz + uz * gry));
    if (kForce) {
        Qxx += ux * Fx; Qyy += uy * Fy; Qzz += uz * Fz;
        Qxy += 0.5f * (ux * Fy + uy * Fx); Qxz += 0.5f * (ux * Fz + uz * Fx); Qyz += 0.5f * (uy * Fz + uz * Fy);
    }
    const float o2 = 1.0f - s2nu, o2b = 1.0f - a.s2b, third = 1.0f / 3.0f;
    const float trQ = Qxx + Qyy + Qzz;
    const float k200 = o2 * (Qxx - trQ * third) + o2b * trQ * third;
    const float k020 = o2 * (Qyy - trQ * third) + o2b * trQ * third;
    const float k002 = o2 * (Qzz - trQ * third) + o2b * trQ * third;
    const float k110 = o2 * Qxy, k101 = o2 * Qxz, k011 = o2 * Qyz;
    const InvAxis Ax(ux), Ay(uy), Az(uz);
    const float g2 = gpx * gpx + gpy * gpy + gpz * gpz;
    const float inv_gm = 1.0f / sqrtf(g2 + a.eps2);
    const float pert = Acoef * inv_gm;
    const float R = a.beta * rr * rb * inv_rho;

    // ---- a_i and b_i, in place, from lambda S = pushed + deferred
    cp_async_wait_all();
#pragma unroll
    for (int c = 0; c < 27; ++c) {
        const float2 P_ = L_s[c * 128], D_ = R_s[c * 128];
        const float lx = P_.x + D_.x, ly = P_.y + D_.y;
        L_s[c * 128] = make_float2((rr * lx + rb * ly) * inv_rho, lx - ly);
    }
    const float a0 = L_s[13 * 128].x, b0 = L_s[13 * 128].y;  // rest direction: cell 13
    const float w0 = 8.0f / 27.0f, k27 = 27.0f / 19.0f;

    // ---- moments of b: the recolouring weight D = sum_i f**_i b_i and the flux direction Q1
    float Dsum, Q1x = 0.0f, Q1y = 0.0f, Q1z = 0.0f;
    {
        float t[27];
#pragma unroll
        for (int c = 0; c < 27; ++c) t[c] = L_s[c * 128].y;
        // Q1 = 27/19 sum_{i>=1} b_i w_i c_i / |c_i|
#pragma unroll
        for (int i = 1; i < 27; ++i) {
            const float v = t[cell(i)] * (k27 * wgt(i) * inv_cnorm(i));
            Q1x += (float)cx(i) * v; Q1y += (float)cy(i) * v; Q1z += (float)cz(i) * v;
        }
        // sum_i b_i h_i = sum_t C_t (psi moments of b)
        float tb[27];
#pragma unroll
        for (int c = 0; c < 27; ++c) tb[c] = t[c];
#pragma unroll
        for (int q = 0; q < 9; ++q) sweep_inv_T(tb[q], tb[9 + q], tb[18 + q], Ax);
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int c = 0; c < 3; ++c) sweep_inv_T(tb[p * 9 + c], tb[p * 9 + 3 + c], tb[p * 9 + 6 + c], Ay);
#pragma unroll
        for (int p = 0; p < 9; ++p) sweep_inv_T(tb[p * 3], tb[p * 3 + 1], tb[p * 3 + 2], Az);
        const float bh = k200 * tb[18] + k020 * tb[6] + k002 * tb[2] + k110 * tb[12] + k101 * tb[10] + k011 * tb[4];
        RawMom B;
        raw_moments(t, B);
        const float B1u = B.m100 * ux + B.m010 * uy + B.m001 * uz;
        float Bux, Buy, Buz;
        m2v(B, ux, uy, uz, Bux, Buy, Buz);
        float B3x, B3y, B3z;
        m3uu(B, ux, uy, uz, B3x, B3y, B3z);
        const float uBu = ux * Bux + uy * Buy + uz * Buz;
        const float B3uuu = ux * B3x + uy * B3y + uz * B3z;
        float Bgx, Bgy, Bgz;
        m2v(B, gpx, gpy, gpz, Bgx, Bgy, Bgz);
        Dsum = rho * fmaf(alpha, b0, k27 * oma * (B.m000 - w0 * b0));
        Dsum = fmaf(rho, 3.0f * B1u + 4.5f * uBu - 1.5f * usq * B.m000 + 4.5f * B3uuu - 4.5f * usq * B1u, Dsum);
        Dsum += -3.0f * nu * ugr * b0 + 9.0f * nu * (grx * Bux + gry * Buy + grz * Buz);
        if (kForce)
            Dsum += 0.5f * (3.0f * (B.m100 * Fx + B.m010 * Fy + B.m001 * Fz) - 3.0f * uF * B.m000 +
                            9.0f * (Fx * Bux + Fy * Buy + Fz * Buz));
        Dsum += bh;
        Dsum = fmaf(pert, gpx * Bgx + gpy * Bgy + gpz * Bgz - g2 * (B.m000 - (2.0f / 3.0f) * b0), Dsum);
    }

    // ---- recolouring: S^r = (rho_r/rho) f** + seg, S^b = (rho_b/rho) f** - seg
    float lrr = Dsum * rb * inv_rho * inv_rho, lrb = -Dsum * rr * inv_rho * inv_rho;
    float lrho = 0.0f;
    const float gQ1 = gpx * Q1x + gpy * Q1y + gpz * Q1z;
    const float lR = oma * gQ1 * inv_gm;
    float lalpha = -R * inv_gm * gQ1;
    lrr = fmaf(lR * a.beta, rb * inv_rho, lrr);
    lrb = fmaf(lR * a.beta, rr * inv_rho, lrb);
    lrho = fmaf(-lR, R * inv_rho, lrho);
    const float sq = R * inv_gm * oma;
    float lgpx = sq * Q1x, lgpy = sq * Q1y, lgpz = sq * Q1z;
    float lgm = -R * lR * inv_gm;

    // ---- moments of a: perturbation, equilibrium, forcing
    float lux, luy, luz, lnu, lgrx, lgry, lgrz, lFx = 0.0f, lFy = 0.0f, lFz = 0.0f, lA;
    {
        float t[27];
#pragma unroll
        for (int c = 0; c < 27; ++c) t[c] = L_s[c * 128].x;
        RawMom A;
        raw_moments(t, A);
        const float sB = A.m000 - (2.0f / 3.0f) * a0;  // sum_i a_i B_i
        float Agx, Agy, Agz, Aux, Auy, Auz, Arx, Ary, Arz;
        m2v(A, gpx, gpy, gpz, Agx, Agy, Agz);
        m2v(A, ux, uy, uz, Aux, Auy, Auz);
        m2v(A, grx, gry, grz, Arx, Ary, Arz);
        // perturbation Omega2_i = A (w_i cgp^2 - B_i |g|^2) / |g|_eps
        lA = (gpx * Agx + gpy * Agy + gpz * Agz - g2 * sB) * inv_gm;
        lgpx = fmaf(2.0f * pert, Agx, lgpx);
        lgpy = fmaf(2.0f * pert, Agy, lgpy);
        lgpz = fmaf(2.0f * pert, Agz, lgpz);
        float lg2 = -pert * sB;
        lgm = fmaf(-lA, pert, lgm);
        lg2 = fmaf(lgm, 0.5f * inv_gm, lg2);
        lgpx = fmaf(2.0f * gpx, lg2, lgpx);
        lgpy = fmaf(2.0f * gpy, lg2, lgpy);
        lgpz = fmaf(2.0f * gpz, lg2, lgpz);
        part[0] += lA * 2.25f / tau;
        // equilibrium f^e_i = rho (varphi_i(alpha) + w_i poly_i(u)) + Phi_i(nu, u, grad rho)
        const float A1u = A.m100 * ux + A.m010 * uy + A.m001 * uz;
        float A3x, A3y, A3z;
        m3uu(A, ux, uy, uz, A3x, A3y, A3z);
        const float uAu = ux * Aux + uy * Auy + uz * Auz;
        const float A3uuu = ux * A3x + uy * A3y + uz * A3z;
        lrho += fmaf(alpha, a0, k27 * oma * (A.m000 - w0 * a0)) + 3.0f * A1u + 4.5f * uAu - 1.5f * usq * A.m000 +
                4.5f * A3uuu - 4.5f * usq * A1u;
        lalpha = fmaf(rho, a0 - k27 * (A.m000 - w0 * a0), lalpha);
        const float c3 = 3.0f - 4.5f * usq, s_u = -3.0f * A.m000 - 9.0f * A1u;
        lux = rho * (c3 * A.m100 + 9.0f * Aux + 13.5f * A3x + ux * s_u);
        luy = rho * (c3 * A.m010 + 9.0f * Auy + 13.5f * A3y + uy * s_u);
        luz = rho * (c3 * A.m001 + 9.0f * Auz + 13.5f * A3z + uz * s_u);
        lnu = -3.0f * a0 * ugr + 9.0f * (ux * Arx + uy * Ary + uz * Arz);
        lux = fmaf(nu, fmaf(-3.0f * a0, grx, 9.0f * Arx), lux);
        luy = fmaf(nu, fmaf(-3.0f * a0, gry, 9.0f * Ary), luy);
        luz = fmaf(nu, fmaf(-3.0f * a0, grz, 9.0f * Arz), luz);
        lgrx = nu * fmaf(-3.0f * a0, ux, 9.0f * Aux);
        lgry = nu * fmaf(-3.0f * a0, uy, 9.0f * Auy);
        lgrz = nu * fmaf(-3.0f * a0, uz, 9.0f * Auz);
        // forcing F'_i = w_i (3 (c_i - u).F + 9 (c_i.u)(c_i.F)), weight 1/2 in f*
        if (kForce) {
            float AFx, AFy, AFz;
            m2v(A, Fx, Fy, Fz, AFx, AFy, AFz);
            lux += 0.5f * (-3.0f * Fx * A.m000 + 9.0f * AFx);
            luy += 0.5f * (-3.0f * Fy * A.m000 + 9.0f * AFy);
            luz += 0.5f * (-3.0f * Fz * A.m000 + 9.0f * AFz);
            lFx = 0.5f * (3.0f * A.m100 - 3.0f * ux * A.m000 + 9.0f * Aux);
            lFy = 0.5f * (3.0f * A.m010 - 3.0f * uy * A.m000 + 9.0f * Auy);
            lFz = 0.5f * (3.0f * A.m001 - 3.0f * uz * A.m000 + 9.0f * Auz);
        }
    }
    // ---- h_i = sum_t C_t psi_t,i(u): lambda_C_t and d/du via the transposed 1-D sweeps
    float l200, l020, l002, l110, l101, l011;
    {
        float lh[27];
#pragma unroll
        for (int c = 0; c < 27; ++c) lh[c] = L_s[c * 128].x;
#pragma unroll
        for (int q = 0; q < 9; ++q) sweep_inv_T(lh[q], lh[9 + q], lh[18 + q], Ax);
#pragma unroll
        for (int a0_ = 0; a0_ < 3; ++a0_)
#pragma unroll
            for (int c = 0; c < 3; ++c) sweep_inv_T(lh[a0_ * 9 + 0 + c], lh[a0_ * 9 + 3 + c], lh[a0_ * 9 + 6 + c], Ay);
#pragma unroll
        for (int p = 0; p < 9; ++p) sweep_inv_T(lh[p * 3 + 0], lh[p * 3 + 1], lh[p * 3 + 2], Az);
#define MM(p, q, r) lh[(p) * 9 + (q) * 3 + (r)]
        l200 = MM(2, 0, 0); l020 = MM(0, 2, 0); l002 = MM(0, 0, 2);
        l110 = MM(1, 1, 0); l101 = MM(1, 0, 1); l011 = MM(0, 1, 1);
        // dG0/du = G1, dG1/du = 2 G2, dG2/du = 0
        lux += k020 * MM(1, 2, 0) + k002 * MM(1, 0, 2) + 2.0f * k110 * MM(2, 1, 0) + 2.0f * k101 * MM(2, 0, 1) + k011 * MM(1, 1, 1);
        luy += k200 * MM(2, 1, 0) + k002 * MM(0, 1, 2) + 2.0f * k110 * MM(1, 2, 0) + k101 * MM(1, 1, 1) + 2.0f * k011 * MM(0, 2, 1);
        luz += k200 * MM(2, 0, 1) + k020 * MM(0, 2, 1) + k110 * MM(1, 1, 1) + 2.0f * k101 * MM(1, 0, 2) + 2.0f * k011 * MM(0, 1, 2);
#undef MM
    }
    // ---- relaxation C = (1 - s2nu) dev Q + (1 - s2b) (tr Q / 3) I
    const float trl = l200 + l020 + l002;
    const float lQxx = o2 * (l200 - trl * third) + o2b * trl * third;
    const float lQyy = o2 * (l020 - trl * third) + o2b * trl * third;
    const float lQzz = o2 * (l002 - trl * third) + o2b * trl * third;
    const float lQxy = o2 * l110, lQxz = o2 * l101, lQyz = o2 * l011;
    const float ls2nu = -(l200 * (Qxx - trQ * third) + l020 * (Qyy - trQ * third) + l002 * (Qzz - trQ * third) +
                          l110 * Qxy + l101 * Qxz + l011 * Qyz);
    // ---- Q: symmetric Lambda (diagonal lQ_aa, off-diagonal lQ_ab / 2)
    const float Lxy = 0.5f * lQxy, Lxz = 0.5f * lQxz, Lyz = 0.5f * lQyz;
    const float Lux = lQxx * ux + Lxy * uy + Lxz * uz;
    const float Luy = Lxy * ux + lQyy * uy + Lyz * uz;
    const float Luz = Lxz * ux + Lyz * uy + lQzz * uz;
    const float Lgx = lQxx * grx + Lxy * gry + Lxz * grz;
    const float Lgy = Lxy * grx + lQyy * gry + Lyz * grz;
    const float Lgz = Lxz * grx + Lyz * gry + lQzz * grz;
    const float Ltr = lQxx + lQyy + lQzz;
    lrho += -(ux * Lux + uy * Luy + uz * Luz) - cs2 * Ltr;
    lux += -2.0f * rho * Lux - nu * (2.0f * Lgx + Ltr * grx);
    luy += -2.0f * rho * Luy - nu * (2.0f * Lgy + Ltr * gry);
    luz += -2.0f * rho * Luz - nu * (2.0f * Lgz + Ltr * grz);
    if (kForce) {
        lux += lQxx * Fx + Lxy * Fy + Lxz * Fz;
        luy += Lxy * Fx + lQyy * Fy + Lyz * Fz;
        luz += Lxz * Fx + Lyz * Fy + lQzz * Fz;
        lFx += Lux; lFy += Luy; lFz += Luz;
    }
    lalpha = fmaf(9.0f / 19.0f * rho, Ltr, lalpha);
    lnu += -(2.0f * (ux * Lgx + uy * Lgy + uz * Lgz) + Ltr * ugr);
    lgrx -= nu * fmaf(2.0f, Lux, Ltr * ux);
    lgry -= nu * fmaf(2.0f, Luy, Ltr * uy);
    lgrz -= nu * fmaf(2.0f, Luz, Ltr * uz);
    // ---- sigma, tau, nu (harmonic mean), alpha-bar
    const float ltau = -lA * Acoef / tau - ls2nu * s2nu * s2nu;
    lnu = fmaf(3.0f, ltau, lnu);
    const float lH = -lnu * nu * nu;
    float lphi = lH * 0.5f * (a.inv_nu_r - a.inv_nu_b);
    part[1] += -lH * hp * a.inv_nu_r * a.inv_nu_r;
    part[2] += -lH * hm * a.inv_nu_b * a.inv_nu_b;
    if (a.alpha_mix) {  // alpha-bar = (rho_r alpha_r + rho_b alpha_b) / rho
        lrr = fmaf(lalpha, (oma - a.oma_r) * inv_rho, lrr);  // (alpha_r - alpha-bar) / rho
        lrb = fmaf(lalpha, (oma - a.oma_b) * inv_rho, lrb);
    } else {
        lphi = fmaf(lalpha, 0.5f * (a.oma_b - a.oma_r), lphi);  // (alpha_r - alpha_b) / 2
    }
    // ---- u = (j + F/2) / rho, F = (rho - rho_b0) g
    const float ljx = lux * inv_rho, ljy = luy * inv_rho, ljz = luz * inv_rho;
    if (kForce) {
        lFx = fmaf(0.5f, ljx, lFx);
        lFy = fmaf(0.5f, ljy, lFy);
        lFz = fmaf(0.5f, ljz, lFz);
        lrho += lFx * a.gx + lFy * a.gy + lFz * a.gz;
    }
    lrho -= (lux * ux + luy * uy + luz * uz) * inv_rho;
    // ---- phi = (A - B)/(A + B), A = rho_r / rho_r0, B = rho_b / rho_b0
    {
        const float S_ = rr * a.inv_rho_r0 + rb * a.inv_rho_b0;
        const float t = lphi / S_;
        lrr = fmaf(t * (1.0f - phi), a.inv_rho_r0, lrr);
        lrb = fmaf(-t * (1.0f + phi), a.inv_rho_b0, lrb);
    }
    lrr += lrho;
    lrb += lrho;

    // ---- outputs: lambda_f_i^k = lambda_j . c_i + c_i Lambda_P c_i + lambda_rho_k, pushed to the
    // slot the pull read (with side walls, W: the reflected direction, selected at run time)
    g.lga[nb.n] = make_float4(lgpx, lgpy, lgpz, lgrx);
    g.lgb[nb.n] = make_float2(lgry, lgrz);
    const AdjPush o{ljx, ljy, ljz, lQxx, lQyy, lQzz, lQxy, lQxz, lQyz, lrr, lrb};
    if (z == 0 || z == N)
        adj_push<W, true>(a, g, nb, z, o);
    else
        adj_push<W, false>(a, g, nb, z, o);
}

#ifndef LBCM_ADJ_MIN_BLOCKS
#define LBCM_ADJ_MIN_BLOCKS 3
#endif
template <bool kForce, bool W>
__global__ void __launch_bounds__(128, LBCM_ADJ_MIN_BLOCKS) adj_collide_kernel(StepArgs a, AdjArgs g) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    extern __shared__ float2 adj_dsm[];  // [2][27][128]: pushed and deferred lambda S(n+1)
    const int t = threadIdx.y * 32 + threadIdx.x;
    float part[3] = {0.0f, 0.0f, 0.0f};
    if (x < a.nx && y < a.ny) adj_collide_node<kForce, W>(a, g, x, y, z, part, adj_dsm + t, adj_dsm + 27 * 128 + t);
    block_accumulate<3>(part, g.acc_coll, block_id());
}

// --------------------------------------------------- transposed gradient stencil (K3)
// lambda_phi(y) = sum over the nodes x whose stencil reads y of 3 w_j c_j . lambda_gphi(x); a
// node x on z = 0 (z = N) reads y through the mirror ghost with c_j's z component flipped,
// except inside the inlet disc, where the ghost is a constant.  Same for rho.  Then
// lambda_rho_k(y) = lambda_phi dphi/drho_k + lambda_rho.
// The 52 neighbour loads are issued in two batches of 13 neighbours before they are used (the
// loop with a use after every load kept few loads in flight and stalled on each); planes away
// from z walls take the stencil's signs at compile time.
template <bool W, bool kZWall>
__device__ __forceinline__ void adj_stencil_sums(const StepArgs &a, const AdjArgs &g, const Nbr &nb, int z,
                                                 float &lphi, float &lrho) {
    const int N = a.nz - 1;
    const bool pz = a.bc_zlo == BC_PERIODIC;
    const bool lo_const = kZWall && !pz && z == 0 && a.bc_zlo == BC_INLET && a.disc[nb.pxy];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float4 A[13];
        float2 B[13];
#pragma unroll
        for (int q = 0; q < 13; ++q) {
            const int src = nb.src(1 + 13 * h + q);  // clamped onto the wall layer: the mirrored reader
            A[q] = __ldg(g.lga + src);
            B[q] = __ldg(g.lgb + src);
        }
#pragma unroll
        for (int q = 0; q < 13; ++q) {
            const int j = 1 + 13 * h + q;
            const bool below = kZWall && !pz && z == 0 && cz(j) == 1;   // x = y - c_j would sit on z = -1
            const bool above = kZWall && !pz && z == N && cz(j) == -1;  // ... on z = N + 1
            // beyond a wall the reader is on this layer and reached y through its mirror ghost
            // with that component of c reversed
            const float czj = (below || above) ? -(float)cz(j) : (float)cz(j);
            const float cxj = W && nb.fx(j) ? -(float)cx(j) : (float)cx(j);
            const float cyj = W && nb.fy(j) ? -(float)cy(j) : (float)cy(j);
            const float w3 = (below && lo_const) ? 0.0f : 3.0f * wgt(j);  // the disc ghost is a constant
            lphi = fmaf(w3, cxj * A[q].x + cyj * A[q].y + czj * A[q].z, lphi);
            lrho = fmaf(w3, cxj * A[q].w + cyj * B[q].x + czj * B[q].y, lrho);
        }
    }
}

template <bool W>
__global__ void __launch_bounds__(128) adj_stencil_kernel(StepArgs a, AdjArgs g) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= a.nx || y >= a.ny) return;
    const Nbr nb(a, x, y, z);
    float lphi = 0.0f, lrho = 0.0f;
    if (a.bc_zlo != BC_PERIODIC && (z == 0 || z == a.nz - 1))
        adj_stencil_sums<W, true>(a, g, nb, z, lphi, lrho);
    else
        adj_stencil_sums<W, false>(a, g, nb, z, lphi, lrho);
    float phv, S_;  // phi and rho_r/rho_r0 + rho_b/rho_b0 of this node
    if (g.mom) {
        const float4 r0 = __ldg(g.mom + nb.n);  // (rho_r, rho_b, sf, jx)
        phv = order_parameter(r0.x, r0.y, a.inv_rho_r0, a.inv_rho_b0);
        S_ = r0.x * a.inv_rho_r0 + r0.y * a.inv_rho_b0;
    } else {
        const float2 ph = __ldg(a.phase + nb.n);  // (phi, rho)
        phv = ph.x;
        S_ = ph.y / (a.rho_r0 * 0.5f * (1.0f + ph.x) + a.rho_b0 * 0.5f * (1.0f - ph.x));
    }
    const float t = lphi / S_;
    g.lr_out[nb.n] = make_float2(fmaf(t * (1.0f - phv), a.inv_rho_r0, lrho), fmaf(-t * (1.0f + phv), a.inv_rho_b0, lrho));
}

// ----------------------------------------------- inlet gradients and outflow transpose
// One warp per (x, y) column, lane i < 27 handling direction i (both colours).
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(128) adj_boundary_kernel(StepArgs a, AdjArgs g) {
    const int lane = threadIdx.x & 31;
    const long long col = (long long)blockIdx.x * 4 + (threadIdx.x >> 5);
    float part[17];
#pragma unroll
    for (int k = 0; k < 17; ++k) part[k] = 0.0f;
    if (col < a.plane) {  // warp-uniform
        const int x = (int)(col % a.nx), y = (int)(col / a.nx);
        const size_t P = (size_t)a.plane, pxy = (size_t)col;
        const int i = lane < 27 ? lane : 0;
        const int cxi = (int)((kPackX >> (2 * i)) & 3ull) - 1, cyi = (int)((kPackY >> (2 * i)) & 3ull) - 1,
                  czi = (int)((kPackZ >> (2 * i)) & 3ull) - 1;
        // source column of the pull of direction i, reflected at free-slip side walls, and the
        // direction that leaves it
        int xs = x - cxi, ys = y - cyi, cxs = cxi, cys = cyi;
        if (xs < 0 || xs >= a.nx) {
            if (a.wall_x) { xs = x; cxs = -cxi; } else xs = wrapi(xs, a.nx);
        }
        if (ys < 0 || ys >= a.ny) {
            if (a.wall_y) { ys = y; cys = -cyi; } else ys = wrapi(ys, a.ny);
        }
        const int ii = dir_of(cxs, cys, czi);
        const int q = cxi * cxi + cyi * cyi + czi * czi;
        const float w_i = q == 0 ? 8.0f / 27.0f : q == 1 ? 2.0f / 27.0f : q == 2 ? 1.0f / 54.0f : 1.0f / 216.0f;
        if (a.bc_zlo == BC_INLET && lane < 27 && czi == 1) {
            if (a.disc[(size_t)ys * a.nx + xs]) {
                // rank of i among the c_z = +1 directions
                int zr = 0;
                for (int j = 0; j < i; ++j) zr += ((int)((kPackZ >> (2 * j)) & 3ull) - 1) == 1;
                const float lam = g.li[(size_t)zr * P + pxy] + g.lr_out[pxy].x;
                InletVel iv;
                inlet_velocity(a.u_in, a.noise_amp, a.fourier, a.xc, a.yc, a.seed, a.step, xs, ys, a.nx, a.ny, iv);
                const float c0 = (float)cxs, c1 = (float)cys, c2 = (float)czi;  // direction leaving the ghost
                const float cu = c0 * iv.ux + c1 * iv.uy + c2 * iv.uz;
                const float usq = iv.ux * iv.ux + iv.uy * iv.uy + iv.uz * iv.uz;
                // d f^e_i / d u = rho_r0 w_i [(3 + 9 cu + 27/2 cu^2 - 9/2 u^2) c_i - (3 + 9 cu) u]
                const float sc = lam * a.rho_r0 * w_i;
                const float dp = fmaf(13.5f * cu, cu, fmaf(9.0f, cu, 3.0f)) - 4.5f * usq;
                const float du = fmaf(-9.0f, cu, -3.0f);
                const float gx_ = sc * fmaf(c0, dp, du * iv.ux);
                const float gy_ = sc * fmaf(c1, dp, du * iv.uy);
                const float gz_ = sc * fmaf(c2, dp, du * iv.uz);
                part[0] = gx_ * iv.dux + gy_ * iv.duy + gz_ * iv.prof;
#pragma unroll
                for (int m = 1; m <= 8; ++m) {
                    part[2 * m - 1] = gz_ * a.u_in * iv.cm[m];
                    part[2 * m] = gz_ * a.u_in * iv.sm[m];
                }
            }
        }
        if (a.bc_zhi == BC_CONVECTIVE) {
            const int N = a.nz - 1, zm = N - 1;
            const Nbr nbm(a, x, y, zm);
            // the source of f_i(x, y, N-1) (plain pull in z: 1 <= N-1; reflected at side walls)
            const int src = nbm.zo[czi + 1] + nbm.yo[cyi + 1] + nbm.xo[cxi + 1];
            float fr = 0.0f, fb = 0.0f;
            if (lane < 27) {  // f(N-1) as the forward step pulled it
                fr = __ldg(g.fm + (size_t)i * P + pxy);
                fb = __ldg(g.fm + (size_t)(27 + i) * P + pxy);
            }
            const float s_ = fr + fb;
            const float rho = warp_sum(s_), jz = warp_sum((float)czi * s_);
            const float Fz = (rho - a.rho_b0) * a.gz;
            const float lam_raw = (jz + 0.5f * Fz) / rho;
            const float lam = fminf(fmaxf(lam_raw, 0.0f), 1.0f);
            const float inv = 1.0f / (1.0f + lam);
            const float2 lrN = g.lr_out[(size_t)N * P + pxy];
            float lvr = 0.0f, lvb = 0.0f, part_l = 0.0f;
            const size_t hr = (size_t)i * P + pxy, hb = (size_t)(27 + i) * P + pxy;
            if (lane < 27) {
                lvr = g.lc[hr] + lrN.x + g.lh_in[hr];
                lvb = g.lc[hb] + lrN.y + g.lh_in[hb];
                g.lh_out[hr] = lvr * inv;
                g.lh_out[hb] = lvb * inv;
                part_l = fmaf(lvr, fr - a.hist_out[hr], lvb * (fb - a.hist_out[hb]));
            }
            const float llam = warp_sum(part_l) * inv;
            if (lane < 27) {
                const bool active = lam_raw > 0.0f && lam_raw < 1.0f;
                const float dl = active ? llam * ((float)czi + 0.5f * a.gz - lam_raw) / rho : 0.0f;
                float2 *slot = g.lp_out + (size_t)ii * a.NN + src;
                float2 v = *slot;
                v.x += fmaf(lvr, lam * inv, dl);
                v.y += fmaf(lvb, lam * inv, dl);
                *slot = v;
            }
        }
    }
    // only blocks holding inlet-disc columns have inlet gradients; the others skip the reduction
    // (the decision is block-uniform, so every thread of a block takes the same branch)
    bool any = false;
#pragma unroll
    for (int k = 0; k < 17; ++k) any |= part[k] != 0.0f;
    if (__syncthreads_or(any)) block_accumulate<17>(part, g.acc_inlet, block_id());
}

// ------------------------------------------------------------------- objectives
// (phi, rho) of a post-collision state: rho_k = sum_i S_i^k.
__global__ void __launch_bounds__(256) obj_fields_kernel(StepArgs a, float2 *ph) {
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < a.NN; n += (long long)gridDim.x * blockDim.x) {
        MassAcc mr, mb;
#pragma unroll
        for (int i = 0; i < 27; ++i) {
            const float2 v = load_pop<STORE_FP32>(a, i, (int)n, no_shift());
            mr.add(i, v.x);
            mb.add(i, v.y);
        }
        const float rr = mr.total(), rb = mb.total();
        ph[n] = make_float2(order_parameter(rr, rb, a.inv_rho_r0, a.inv_rho_b0), rr + rb);
    }
}

// Interface area sum over 1 <= z <= nz-2 of sqrt(|grad phi|^2 + eps^2) (isotropic stencil,
// periodic in x and y); writes lambda_grad phi = grad phi / sqrt(...) (zero elsewhere).
__global__ void __launch_bounds__(128) obj_area_kernel(StepArgs a, const float2 *ph, float4 *lga, float2 *lgb,
                                                      double *acc, float eps2) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    float part[1] = {0.0f};
    if (x < a.nx && y < a.ny) {
        const Nbr nb(a, x, y, z);
        float gx = 0.0f, gy = 0.0f, gz = 0.0f;
        const bool inside = z >= 1 && z <= a.nz - 2;
        if (inside) {
#pragma unroll
            for (int j = 1; j < 27; j += 2) {
                const float w3 = 3.0f * wgt(j);
                const float d = __ldg(ph + nb.nbr(j)).x - __ldg(ph + nb.nbr(j + 1)).x;
                gx = fmaf(w3 * cx(j), d, gx);
                gy = fmaf(w3 * cy(j), d, gy);
                gz = fmaf(w3 * cz(j), d, gz);
            }
            const float m = sqrtf(gx * gx + gy * gy + gz * gz + eps2);
            part[0] = m;
            const float im = 1.0f / m;
            gx *= im; gy *= im; gz *= im;
        }
        lga[nb.n] = make_float4(gx, gy, gz, 0.0f);
        lgb[nb.n] = make_float2(0.0f, 0.0f);
    }
    block_accumulate<1>(part, acc, block_id());
}

// Penetration length (smooth maximum): L = delta log sum_n H(phi_n) exp(z_n / delta) with the
// redness weight H = ((1 + phi)/2)^2, accumulated as sum H exp((z - N) / delta).
__global__ void __launch_bounds__(128) obj_pen_sum_kernel(StepArgs a, const float2 *ph, double *acc, float inv_delta) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    float part[1] = {0.0f};
    if (x < a.nx && y < a.ny) {
        const float h = 0.5f * (1.0f + __ldg(ph + ((size_t)z * a.plane + (size_t)y * a.nx + x)).x);
        part[0] = h * h * expf((float)(z - (a.nz - 1)) * inv_delta);
    }
    block_accumulate<1>(part, acc, block_id());
}

// lambda_S(T)(n, k, i) = dL/dphi_n dphi/drho_k for every i; clears the deferred part.
__global__ void __launch_bounds__(256) obj_pen_adjoint_kernel(StepArgs a, const float2 *ph, const double *Z,
                                                             float2 *lp, float2 *lr, float inv_delta, float delta) {
    const float inv_Z = (float)(1.0 / *Z);
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < a.NN; n += (long long)gridDim.x * blockDim.x) {
        const float2 v = ph[n];
        const int z = (int)(n / a.plane);
        const float lphi = delta * 0.5f * (1.0f + v.x) * expf((float)(z - (a.nz - 1)) * inv_delta) * inv_Z;
        const float S_ = v.y / (a.rho_r0 * 0.5f * (1.0f + v.x) + a.rho_b0 * 0.5f * (1.0f - v.x));
        const float q = lphi / S_;
        const float2 o = make_float2(q * (1.0f - v.x) * a.inv_rho_r0, -q * (1.0f + v.x) * a.inv_rho_b0);
#pragma unroll
        for (int i = 0; i < 27; ++i) lp[(size_t)i * a.NN + n] = o;
        lr[n] = make_float2(0.0f, 0.0f);
    }
}

// lambda_S(T)(n, k, i) = lr_obj(n, k) for every i (density adjoint of the objective).
__global__ void __launch_bounds__(256) obj_fill_kernel(long long NN, const float2 *lr_obj, float2 *lp, float2 *lr) {
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < NN; n += (long long)gridDim.x * blockDim.x) {
        const float2 o = lr_obj[n];
#pragma unroll
        for (int i = 0; i < 27; ++i) lp[(size_t)i * NN + n] = o;
        lr[n] = make_float2(0.0f, 0.0f);
    }
}

// out[k] = sum_b acc[b * nv + k0 + k] (FP64, fixed order: deterministic).
__global__ void __launch_bounds__(1024) adj_reduce_kernel(const double *acc, long long nblk, int nv, int k0,
                                                         double *out) {
    __shared__ double sh[1024];
    const int k = blockIdx.x;
    double s = 0.0;
    for (long long b = threadIdx.x; b < nblk; b += blockDim.x) s += acc[b * nv + k0 + k];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = sh[0];
}

// J of the penetration objective from Z: L = N + delta log Z.
__global__ void obj_pen_value_kernel(const double *Z, double *out, double N, double delta) {
    if (threadIdx.x == 0 && blockIdx.x == 0) out[0] = N + delta * log(*Z);
}

// dJ/dS(n) in the canonical layout [k][i][z][y][x] from the split adjoint state.
__global__ void __launch_bounds__(256) adj_state_kernel(StepArgs a, AdjArgs g, float *out) {
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < a.NN; n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % a.nx), y = (int)((n / a.nx) % a.ny), z = (int)(n / a.plane);
        const Nbr nb(a, x, y, z);
        const bool own_in_disc = a.bc_zlo == BC_INLET && z == 0 && a.disc[nb.pxy];
#pragma unroll
        for (int i = 0; i < 27; ++i) {
            const float2 v = adj_slot(a, g, nb, i, z, own_in_disc);
            out[(size_t)i * a.NN + n] = v.x;
            out[(size_t)(27 + i) * a.NN + n] = v.y;
        }
    }
}

// ------------------------------------------------------------------------ launchers
static dim3 node_block() { return dim3(32, 4, 1); }
static dim3 node_grid(const StepArgs &a) { return dim3((a.nx + 31) / 32, (a.ny + 3) / 4, a.nz); }
static dim3 col_block() { return dim3(128, 1, 1); }  // four columns, one warp each
static dim3 col_grid(const StepArgs &a) { return dim3((unsigned)((a.plane + 3) / 4), 1, 1); }

long long adj_collide_blocks(const StepArgs &a) {
    const dim3 gr = node_grid(a);
    return (long long)gr.x * gr.y * gr.z;
}
long long adj_boundary_blocks(const StepArgs &a) {
    const dim3 gr = col_grid(a);
    return (long long)gr.x * gr.y * gr.z;
}

constexpr int kAdjSmem = 2 * 27 * 128 * (int)sizeof(float2);

cudaError_t launch_adjoint_step(const StepArgs &a, const AdjArgs &g, cudaStream_t s, long long *launches) {
    const bool force = a.gx != 0.0f || a.gy != 0.0f || a.gz != 0.0f;
    const bool walls = a.wall_x || a.wall_y;
    static bool attr = false;  // the dynamic shared memory exceeds the 48 KB default
    if (!attr) {
        cudaFuncSetAttribute(adj_collide_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kAdjSmem);
        cudaFuncSetAttribute(adj_collide_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kAdjSmem);
        cudaFuncSetAttribute(adj_collide_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kAdjSmem);
        cudaFuncSetAttribute(adj_collide_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kAdjSmem);
        attr = true;
    }
    const dim3 gr = node_grid(a), bl = node_block();
    if (force && walls)
        adj_collide_kernel<true, true><<<gr, bl, kAdjSmem, s>>>(a, g);
    else if (force)
        adj_collide_kernel<true, false><<<gr, bl, kAdjSmem, s>>>(a, g);
    else if (walls)
        adj_collide_kernel<false, true><<<gr, bl, kAdjSmem, s>>>(a, g);
    else
        adj_collide_kernel<false, false><<<gr, bl, kAdjSmem, s>>>(a, g);
    if (walls)
        adj_stencil_kernel<true><<<gr, bl, 0, s>>>(a, g);
    else
        adj_stencil_kernel<false><<<gr, bl, 0, s>>>(a, g);
    *launches += 2;
    if (a.bc_zlo == BC_INLET || a.bc_zhi == BC_CONVECTIVE) {
        adj_boundary_kernel<<<col_grid(a), col_block(), 0, s>>>(a, g);
        *launches += 1;
    }
    return cudaGetLastError();
}

static int stride_grid(long long n) {
    long long b = (n + 255) / 256;
    return (int)std::min<long long>(std::max<long long>(b, 1), 152ll * 32);
}

cudaError_t launch_objective(const StepArgs &a, const AdjArgs &g, int objective, const double *args, float2 *ph,
                             float2 *lr_obj, double *acc_obj, double *scalar, cudaStream_t s, long long *launches) {
    const long long nblk = adj_collide_blocks(a);
    obj_fields_kernel<<<stride_grid(a.NN), 256, 0, s>>>(a, ph);
    *launches += 1;
    if (objective == 0) {  // interface area
        AdjArgs o = g;
        o.lr_out = lr_obj;
        StepArgs ao = a;
        ao.phase = ph;
        const float eps = (float)args[0];
        obj_area_kernel<<<node_grid(a), node_block(), 0, s>>>(a, ph, g.lga, g.lgb, acc_obj, eps * eps);
        if (a.wall_x || a.wall_y)
            adj_stencil_kernel<true><<<node_grid(a), node_block(), 0, s>>>(ao, o);
        else
            adj_stencil_kernel<false><<<node_grid(a), node_block(), 0, s>>>(ao, o);
        obj_fill_kernel<<<stride_grid(a.NN), 256, 0, s>>>(a.NN, lr_obj, g.lp_out, g.lr_out);
        adj_reduce_kernel<<<1, 1024, 0, s>>>(acc_obj, nblk, 1, 0, scalar);
        *launches += 4;
    } else {  // penetration length
        const double delta = args[0];
        obj_pen_sum_kernel<<<node_grid(a), node_block(), 0, s>>>(a, ph, acc_obj, (float)(1.0 / delta));
        adj_reduce_kernel<<<1, 1024, 0, s>>>(acc_obj, nblk, 1, 0, scalar + 1);
        obj_pen_value_kernel<<<1, 32, 0, s>>>(scalar + 1, scalar, (double)(a.nz - 1), delta);
        obj_pen_adjoint_kernel<<<stride_grid(a.NN), 256, 0, s>>>(a, ph, scalar + 1, g.lp_out, g.lr_out,
                                                                 (float)(1.0 / delta), (float)delta);
        *launches += 4;
    }
    return cudaGetLastError();
}

cudaError_t launch_adjoint_reduce(const AdjArgs &g, long long nblk_coll, long long nblk_inlet, double *out,
                                  cudaStream_t s, long long *launches) {
    // out[1] = u_in, out[2..4] = sigma, nu_r, nu_b, out[5..20] = a_1, b_1, ..., a_8, b_8
    adj_reduce_kernel<<<1, 1024, 0, s>>>(g.acc_inlet, nblk_inlet, 17, 0, out + 1);
    adj_reduce_kernel<<<3, 1024, 0, s>>>(g.acc_coll, nblk_coll, 3, 0, out + 2);
    adj_reduce_kernel<<<16, 1024, 0, s>>>(g.acc_inlet, nblk_inlet, 17, 1, out + 5);
    *launches += 3;
    return cudaGetLastError();
}

cudaError_t launch_adjoint_state(const StepArgs &a, const AdjArgs &g, float *out, cudaStream_t s, long long *launches) {
    adj_state_kernel<<<stride_grid(a.NN), 256, 0, s>>>(a, g, out);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace lbcm
