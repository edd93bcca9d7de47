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

// Adds the block sums of v[0..NV) (FP64) to acc[blk * NV + k].  Every thread of the block
// must call it (no early return before).
template <int NV>
__device__ __forceinline__ void block_accumulate(const float (&v)[NV], double *acc, long long blk) {
    __shared__ double sh[NV][32];
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int lane = tid & 31, warp = tid >> 5, nwarp = (nthr + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double d = (double)v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
        if (lane == 0) sh[k][warp] = d;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double d = lane < nwarp ? sh[k][lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
            if (lane == 0) acc[blk * NV + k] += d;
        }
    }
}

__device__ __forceinline__ long long block_id() {
    return blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
}

// lambda_S(n+1) of slot (node nb.n, direction i): the pushed part plus the deferred density
// adjoint of the node that reads the slot in step n+1, if a pull reads it (the inlet disc and
// the convective plane read nothing).
__device__ __forceinline__ float2 adj_slot(const StepArgs &a, const AdjArgs &g, const Nbr &nb, int i, int z,
                                           bool own_in_disc) {
    float2 v = __ldg(g.lp_in + (size_t)i * a.NN + nb.n);
    bool read = true;
    if (a.bc_zlo != BC_PERIODIC) {
        const int zr = z + cz(i);
        if (a.bc_zhi == BC_CONVECTIVE && zr >= a.nz - 1) read = false;
        if (zr < 0 && own_in_disc) read = false;
    }
    if (read) {
        const float2 r = __ldg(g.lr_in + nb.nbr(i));
        v.x += r.x;
        v.y += r.y;
    }
    return v;
}

// 1-D transpose of the inverse sweep: M_a = sum_c v_c G_a[c](u) for a = 0, 1, 2.
__device__ __forceinline__ void sweep_inv_T(float &a0, float &a1, float &a2, const InvAxis &A) {
    const float v0 = a0, v1 = a1, v2 = a2;
    a0 = fmaf(A.g0[0], v0, fmaf(A.g0[1], v1, A.g0[2] * v2));
    a1 = fmaf(A.g1[0], v0, fmaf(A.g1[1], v1, A.g1[2] * v2));
    a2 = fmaf(0.5f, v0 + v2, -v1);
}

// ---------------------------------------------------------------- reverse collision
template <bool kForce>
__device__ __forceinline__ void adj_collide_node(const StepArgs &a, const AdjArgs &g, int x, int y, int z,
                                                 float (&part)[3]) {
    const Nbr nb(a, x, y, z);
    const int N = a.nz - 1;
    const bool pz = a.bc_zlo == BC_PERIODIC;
    const bool conv_top = !pz && z == N && a.bc_zhi == BC_CONVECTIVE;
    const bool own_in_disc = !pz && z == 0 && a.bc_zlo == BC_INLET && a.disc[nb.pxy];

    // ---- forward recomputation (as collide_from_moments, moments of order <= 2)
    Moments mo;
    gather_moments<STORE_FP32>(a, nb, z, mo);
    float gpx, gpy, gpz, grx, gry, grz;
    stencil_gradients<STORE_FP32>(a, nb, z, gpx, gpy, gpz, grx, gry, grz);
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
    const float alpha = hp * a.alpha_r + hm * a.alpha_b, oma = 1.0f - alpha;
    const float nu = 1.0f / (hp * a.inv_nu_r + hm * a.inv_nu_b);
    const float tau = 3.0f * nu + 0.5f, s2nu = 1.0f / tau;
    const float Acoef = 2.25f * a.sigma / tau;
    const float usq = ux * ux + uy * uy + uz * uz;
    const float ugr = ux * grx + uy * gry + uz * grz;
    const float uF = ux * Fx + uy * Fy + uz * Fz;
    const float cs2 = oma * (9.0f / 19.0f);
    // Q = Pi(f) - Pi(f^e) + Pi(F')/2 - rho u u terms: the second central moment of f - f^e + F'/2
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
    float V00[3], V10[3], V01[3], V20[3], V02[3], V11[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        V00[c] = g2c(c - 1) * k002;
        V10[c] = Az.g1[c] * k101;
        V01[c] = Az.g1[c] * k011;
        V20[c] = Az.g0[c] * k200;
        V02[c] = Az.g0[c] * k020;
        V11[c] = Az.g0[c] * k110;
    }
    float W0[3][3], W1[3][3], W2[3][3];
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            W0[b][c] = fmaf(Ay.g0[b], V00[c], fmaf(Ay.g1[b], V01[c], g2c(b - 1) * V02[c]));
            W1[b][c] = fmaf(Ay.g0[b], V10[c], Ay.g1[b] * V11[c]);
            W2[b][c] = Ay.g0[b] * V20[c];
        }
    const float g2 = gpx * gpx + gpy * gpy + gpz * gpz;
    const float inv_gm = 1.0f / sqrtf(g2 + a.eps2);
    const float pert = Acoef * inv_gm;
    const float R = a.beta * rr * rb * inv_rho;

    // ---- pass over the directions: lambda of S(n+1) -> lambda of f** and of the recolouring
    float lh[27];  // lambda of f* (= of f^e, h and the perturbation; F'/2 takes half)
    float l_xr = 0.0f, l_xb = 0.0f;                       // lambda of rho_r/rho, rho_b/rho
    float s_fe = 0.0f, s_dvp = 0.0f, s_u = 0.0f, s_nu = 0.0f, s_pert = 0.0f, s_B = 0.0f, s_w = 0.0f;
    float v_dp[3] = {0, 0, 0}, v_nug[3] = {0, 0, 0}, v_nuu[3] = {0, 0, 0}, v_pgp[3] = {0, 0, 0};
    float v_wcF[3] = {0, 0, 0}, v_wcu[3] = {0, 0, 0}, v_wc[3] = {0, 0, 0};
    float s_bcv = 0.0f, s_bcd = 0.0f, v_seg[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        const float c0 = (float)cx(i), c1 = (float)cy(i), c2 = (float)cz(i);
        const float cu = c0 * ux + c1 * uy + c2 * uz;
        const float cgr = c0 * grx + c1 * gry + c2 * grz;
        const float cgp = c0 * gpx + c1 * gpy + c2 * gpz;
        const float vp = varphi(i, alpha, oma);
        const float dvp = csq(i) == 0 ? 1.0f : -varphi_k(i);
        const float pl = eq_poly(cu, usq);
        const float Phi = csq(i) == 0 ? -3.0f * nu * ugr : phi_corr(i) * nu * cu * cgr;
        const float fe = rho * fmaf(wgt(i), pl, vp) + Phi;
        float fs = fe;
        float cF = 0.0f;
        if (kForce) {
            cF = c0 * Fx + c1 * Fy + c2 * Fz;
            fs += 0.5f * wgt(i) * (3.0f * (cF - uF) + 9.0f * cu * cF);
        }
        const int X = cx(i) + 1, Y = cy(i) + 1, Z = cz(i) + 1;
        fs += fmaf(Ax.g0[X], W0[Y][Z], fmaf(Ax.g1[X], W1[Y][Z], g2c(cx(i)) * W2[Y][Z]));
        const float pq = wgt(i) * cgp * cgp - bcoef(i) * g2;
        const float fss = fmaf(pert, pq, fs);
        const float2 L = adj_slot(a, g, nb, i, z, own_in_disc);
        l_xr = fmaf(fss, L.x, l_xr);
        l_xb = fmaf(fss, L.y, l_xb);
        const float ai = (rr * L.x + rb * L.y) * inv_rho;
        lh[cell(i)] = ai;
        // recolouring flux seg_i = R cos_i varphi_i, cos_i = cgp / (|c_i| |g|)
        if (csq(i) != 0) {
            const float bi = L.x - L.y;
            const float t = bi * inv_cnorm(i);
            s_bcv = fmaf(t * cgp, vp, s_bcv);
            s_bcd = fmaf(t * cgp, dvp, s_bcd);
            v_seg[0] += c0 * t * vp; v_seg[1] += c1 * t * vp; v_seg[2] += c2 * t * vp;
        }
        // perturbation
        s_pert = fmaf(ai, pq, s_pert);
        s_B = fmaf(ai, bcoef(i), s_B);
        const float awg = ai * wgt(i) * cgp;
        v_pgp[0] += c0 * awg; v_pgp[1] += c1 * awg; v_pgp[2] += c2 * awg;
        // equilibrium
        s_fe = fmaf(ai, fmaf(wgt(i), pl, vp), s_fe);
        s_dvp = fmaf(ai, dvp, s_dvp);
        const float aw = ai * wgt(i);
        const float dpl = fmaf(13.5f * cu, cu, fmaf(9.0f, cu, 3.0f)) - 4.5f * usq;
        v_dp[0] += c0 * aw * dpl; v_dp[1] += c1 * aw * dpl; v_dp[2] += c2 * aw * dpl;
        s_u = fmaf(aw, fmaf(-9.0f, cu, -3.0f), s_u);
        if (csq(i) != 0) {
            const float ap = ai * phi_corr(i);
            s_nu = fmaf(ap * cu, cgr, s_nu);
            v_nug[0] += c0 * ap * cgr; v_nug[1] += c1 * ap * cgr; v_nug[2] += c2 * ap * cgr;
            v_nuu[0] += c0 * ap * cu; v_nuu[1] += c1 * ap * cu; v_nuu[2] += c2 * ap * cu;
        }
        if (kForce) {
            s_w += aw;
            v_wcF[0] += c0 * aw * cF; v_wcF[1] += c1 * aw * cF; v_wcF[2] += c2 * aw * cF;
            v_wcu[0] += c0 * aw * cu; v_wcu[1] += c1 * aw * cu; v_wcu[2] += c2 * aw * cu;
            v_wc[0] += c0 * aw; v_wc[1] += c1 * aw; v_wc[2] += c2 * aw;
        }
    }
    const float a0 = lh[cell(0)];

    // ---- recolouring: S^r = (rho_r/rho) f** + seg, S^b = (rho_b/rho) f** - seg
    float lrr = l_xr * inv_rho, lrb = l_xb * inv_rho;
    float lrho = -(l_xr * rr + l_xb * rb) * inv_rho * inv_rho;
    const float lR = s_bcv * inv_gm;
    float lalpha = R * inv_gm * s_bcd;
    lrr = fmaf(lR * a.beta, rb * inv_rho, lrr);
    lrb = fmaf(lR * a.beta, rr * inv_rho, lrb);
    lrho = fmaf(-lR, R * inv_rho, lrho);
    float lgpx = R * inv_gm * v_seg[0], lgpy = R * inv_gm * v_seg[1], lgpz = R * inv_gm * v_seg[2];
    float lgm = -R * lR * inv_gm;
    // ---- perturbation: Omega2_i = A (w_i cgp^2 - B_i |g|^2) / |g|_eps
    const float lA = s_pert * inv_gm;
    lgpx = fmaf(2.0f * pert, v_pgp[0], lgpx);
    lgpy = fmaf(2.0f * pert, v_pgp[1], lgpy);
    lgpz = fmaf(2.0f * pert, v_pgp[2], lgpz);
    float lg2 = -pert * s_B;
    lgm = fmaf(-lA, pert, lgm);
    lg2 = fmaf(lgm, 0.5f * inv_gm, lg2);
    lgpx = fmaf(2.0f * gpx, lg2, lgpx);
    lgpy = fmaf(2.0f * gpy, lg2, lgpy);
    lgpz = fmaf(2.0f * gpz, lg2, lgpz);
    // ---- equilibrium f^e_i = rho (varphi_i(alpha) + w_i poly_i(u)) + Phi_i(nu, u, grad rho)
    lrho += s_fe;
    lalpha = fmaf(rho, s_dvp, lalpha);
    float lux = rho * fmaf(ux, s_u, v_dp[0]);
    float luy = rho * fmaf(uy, s_u, v_dp[1]);
    float luz = rho * fmaf(uz, s_u, v_dp[2]);
    float lnu = fmaf(-3.0f * a0, ugr, s_nu);
    lux = fmaf(nu, fmaf(-3.0f * a0, grx, v_nug[0]), lux);
    luy = fmaf(nu, fmaf(-3.0f * a0, gry, v_nug[1]), luy);
    luz = fmaf(nu, fmaf(-3.0f * a0, grz, v_nug[2]), luz);
    float lgrx = nu * fmaf(-3.0f * a0, ux, v_nuu[0]);
    float lgry = nu * fmaf(-3.0f * a0, uy, v_nuu[1]);
    float lgrz = nu * fmaf(-3.0f * a0, uz, v_nuu[2]);
    // ---- forcing F'_i = w_i (3 (c_i - u).F + 9 (c_i.u)(c_i.F)), weight 1/2 in f*
    float lFx = 0.0f, lFy = 0.0f, lFz = 0.0f;
    if (kForce) {
        lux += 0.5f * (-3.0f * Fx * s_w + 9.0f * v_wcF[0]);
        luy += 0.5f * (-3.0f * Fy * s_w + 9.0f * v_wcF[1]);
        luz += 0.5f * (-3.0f * Fz * s_w + 9.0f * v_wcF[2]);
        lFx = 0.5f * (3.0f * v_wc[0] - 3.0f * ux * s_w + 9.0f * v_wcu[0]);
        lFy = 0.5f * (3.0f * v_wc[1] - 3.0f * uy * s_w + 9.0f * v_wcu[1]);
        lFz = 0.5f * (3.0f * v_wc[2] - 3.0f * uz * s_w + 9.0f * v_wcu[2]);
    }
    // ---- h_i = sum_t C_t psi_t,i(u): lambda_C_t and d/du via the transposed 1-D sweeps
    // M[a][b][c] = sum_i lh_i G_a[cx](ux) G_b[cy](uy) G_c[cz](uz)
#pragma unroll
    for (int q = 0; q < 9; ++q) sweep_inv_T(lh[q], lh[9 + q], lh[18 + q], Ax);
#pragma unroll
    for (int a0_ = 0; a0_ < 3; ++a0_)
#pragma unroll
        for (int c = 0; c < 3; ++c) sweep_inv_T(lh[a0_ * 9 + 0 + c], lh[a0_ * 9 + 3 + c], lh[a0_ * 9 + 6 + c], Ay);
#pragma unroll
    for (int p = 0; p < 9; ++p) sweep_inv_T(lh[p * 3 + 0], lh[p * 3 + 1], lh[p * 3 + 2], Az);
#define MM(p, q, r) lh[(p) * 9 + (q) * 3 + (r)]
    const float l200 = MM(2, 0, 0), l020 = MM(0, 2, 0), l002 = MM(0, 0, 2);
    const float l110 = MM(1, 1, 0), l101 = MM(1, 0, 1), l011 = MM(0, 1, 1);
    // dG0/du = G1, dG1/du = 2 G2, dG2/du = 0
    lux += k020 * MM(1, 2, 0) + k002 * MM(1, 0, 2) + 2.0f * k110 * MM(2, 1, 0) + 2.0f * k101 * MM(2, 0, 1) + k011 * MM(1, 1, 1);
    luy += k200 * MM(2, 1, 0) + k002 * MM(0, 1, 2) + 2.0f * k110 * MM(1, 2, 0) + k101 * MM(1, 1, 1) + 2.0f * k011 * MM(0, 2, 1);
    luz += k200 * MM(2, 0, 1) + k020 * MM(0, 2, 1) + k110 * MM(1, 1, 1) + 2.0f * k101 * MM(1, 0, 2) + 2.0f * k011 * MM(0, 1, 2);
#undef MM
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
    part[0] += lA * 2.25f / tau;
    const float ltau = -lA * Acoef / tau - ls2nu * s2nu * s2nu;
    lnu = fmaf(3.0f, ltau, lnu);
    const float lH = -lnu * nu * nu;
    float lphi = lH * 0.5f * (a.inv_nu_r - a.inv_nu_b);
    part[1] += -lH * hp * a.inv_nu_r * a.inv_nu_r;
    part[2] += -lH * hm * a.inv_nu_b * a.inv_nu_b;
    lphi = fmaf(lalpha, 0.5f * (a.alpha_r - a.alpha_b), lphi);
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

    // ---- outputs: lambda_f_i^k = lambda_j . c_i + c_i Lambda_P c_i + lambda_rho_k, pushed
    g.lga[nb.n] = make_float4(lgpx, lgpy, lgpz, lgrx);
    g.lgb[nb.n] = make_float2(lgry, lgrz);
    const size_t P = (size_t)a.plane;
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        const float c0 = (float)cx(i), c1 = (float)cy(i), c2 = (float)cz(i);
        float lf = c0 * ljx + c1 * ljy + c2 * ljz;
        lf += c0 * c0 * lQxx + c1 * c1 * lQyy + c2 * c2 * lQzz + c0 * c1 * lQxy + c0 * c2 * lQxz + c1 * c2 * lQyz;
        const float2 o = make_float2(lf + lrr, lf + lrb);
        if (conv_top) {
            // f(N) comes from the outflow rule: its adjoint goes to the boundary kernel; the
            // slots the plain pulls would have read are read by nobody
            g.lc[(size_t)i * P + nb.pxy] = o.x;
            g.lc[(size_t)(27 + i) * P + nb.pxy] = o.y;
            if (cz(i) >= 0) g.lp_out[(size_t)i * a.NN + nb.src(i)] = make_float2(0.0f, 0.0f);
            if (cz(i) == 1) g.lp_out[(size_t)i * a.NN + nb.n] = make_float2(0.0f, 0.0f);
        } else if (!pz && z == 0 && cz(i) == 1) {
            const int xs = nb.xo[cx(i) + 1], ys = nb.yo[cy(i) + 1];  // source column (offsets)
            const size_t slot = (size_t)mirror_z(i) * a.NN + ys + xs;
            if (a.bc_zlo == BC_INLET && a.disc[ys + xs]) {
                g.li[(size_t)zrank(i) * P + nb.pxy] = o.x;
                g.lp_out[slot] = make_float2(0.0f, 0.0f);
            } else {
                g.lp_out[slot] = o;
            }
        } else if (!pz && z == N && cz(i) == -1 && a.bc_zhi == BC_FREESLIP) {
            const int xs = nb.xo[cx(i) + 1], ys = nb.yo[cy(i) + 1];
            g.lp_out[(size_t)mirror_z(i) * a.NN + (size_t)N * P + ys + xs] = o;
        } else {
            g.lp_out[(size_t)i * a.NN + nb.src(i)] = o;
        }
    }
}

template <bool kForce>
__global__ void __launch_bounds__(128) adj_collide_kernel(StepArgs a, AdjArgs g) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    float part[3] = {0.0f, 0.0f, 0.0f};
    if (x < a.nx && y < a.ny) adj_collide_node<kForce>(a, g, x, y, z, part);
    block_accumulate<3>(part, g.acc_coll, block_id());
}

// --------------------------------------------------- transposed gradient stencil (K3)
// lambda_phi(y) = sum over the nodes x whose stencil reads y of 3 w_j c_j . lambda_gphi(x); a
// node x on z = 0 (z = N) reads y through the mirror ghost with c_j's z component flipped,
// except inside the inlet disc, where the ghost is a constant.  Same for rho.  Then
// lambda_rho_k(y) = lambda_phi dphi/drho_k + lambda_rho.
__global__ void __launch_bounds__(128) adj_stencil_kernel(StepArgs a, AdjArgs g) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= a.nx || y >= a.ny) return;
    const Nbr nb(a, x, y, z);
    const int N = a.nz - 1;
    const bool pz = a.bc_zlo == BC_PERIODIC;
    const bool lo_const = !pz && z == 0 && a.bc_zlo == BC_INLET && a.disc[nb.pxy];
    float lphi = 0.0f, lrho = 0.0f;
#pragma unroll
    for (int j = 1; j < 27; ++j) {
        const bool below = !pz && z == 0 && cz(j) == 1;   // x = y - c_j would sit on z = -1
        const bool above = !pz && z == N && cz(j) == -1;  // ... on z = N + 1
        if (below && lo_const) continue;
        const float czj = (below || above) ? -(float)cz(j) : (float)cz(j);
        const int src = nb.src(j);  // clamped onto the wall plane: the mirrored reader
        const float4 A = __ldg(g.lga + src);
        const float2 B = __ldg(g.lgb + src);
        const float w3 = 3.0f * wgt(j);
        lphi = fmaf(w3, (float)cx(j) * A.x + (float)cy(j) * A.y + czj * A.z, lphi);
        lrho = fmaf(w3, (float)cx(j) * A.w + (float)cy(j) * B.x + czj * B.y, lrho);
    }
    const float2 ph = __ldg(a.phase + nb.n);  // (phi, rho) of this node
    const float S_ = ph.y / (a.rho_r0 * 0.5f * (1.0f + ph.x) + a.rho_b0 * 0.5f * (1.0f - ph.x));
    const float t = lphi / S_;
    g.lr_out[nb.n] = make_float2(fmaf(t * (1.0f - ph.x), a.inv_rho_r0, lrho), fmaf(-t * (1.0f + ph.x), a.inv_rho_b0, lrho));
}

// ----------------------------------------------- inlet gradients and outflow transpose
__global__ void __launch_bounds__(256) adj_boundary_kernel(StepArgs a, AdjArgs g) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    float part[17];
#pragma unroll
    for (int k = 0; k < 17; ++k) part[k] = 0.0f;
    if (x < a.nx && y < a.ny) {
        const size_t P = (size_t)a.plane, pxy = (size_t)y * a.nx + x;
        if (a.bc_zlo == BC_INLET) {
            const float lrr0 = g.lr_out[pxy].x;  // deferred red density adjoint of (x, y, 0)
#pragma unroll
            for (int i = 0; i < 27; ++i) {
                if (cz(i) != 1) continue;
                const int xs = wrapi(x - cx(i), a.nx), ys = wrapi(y - cy(i), a.ny);
                if (!a.disc[(size_t)ys * a.nx + xs]) continue;
                const float lam = g.li[(size_t)zrank(i) * P + pxy] + lrr0;
                InletVel iv;
                inlet_velocity(a.u_in, a.noise_amp, a.fourier, a.xc, a.yc, a.seed, a.step, xs, ys, a.nx, a.ny, iv);
                const float c0 = (float)cx(i), c1 = (float)cy(i), c2 = (float)cz(i);
                const float cu = c0 * iv.ux + c1 * iv.uy + c2 * iv.uz;
                const float usq = iv.ux * iv.ux + iv.uy * iv.uy + iv.uz * iv.uz;
                // d f^e_i / d u = rho_r0 w_i [(3 + 9 cu + 27/2 cu^2 - 9/2 u^2) c_i - (3 + 9 cu) u]
                const float sc = lam * a.rho_r0 * wgt(i);
                const float dp = fmaf(13.5f * cu, cu, fmaf(9.0f, cu, 3.0f)) - 4.5f * usq;
                const float du = fmaf(-9.0f, cu, -3.0f);
                const float gx_ = sc * fmaf(c0, dp, du * iv.ux);
                const float gy_ = sc * fmaf(c1, dp, du * iv.uy);
                const float gz_ = sc * fmaf(c2, dp, du * iv.uz);
                part[0] += gx_ * iv.dux + gy_ * iv.duy + gz_ * iv.prof;
#pragma unroll
                for (int m = 1; m <= 8; ++m) {
                    part[2 * m - 1] = fmaf(gz_ * a.u_in, iv.cm[m], part[2 * m - 1]);
                    part[2 * m] = fmaf(gz_ * a.u_in, iv.sm[m], part[2 * m]);
                }
            }
        }
        if (a.bc_zhi == BC_CONVECTIVE) {
            const int N = a.nz - 1, zm = N - 1;
            const Nbr nbm(a, x, y, zm);
            float fr[27], fb[27];
            float rho = 0.0f, jz = 0.0f;
#pragma unroll
            for (int i = 0; i < 27; ++i) {
                const float2 v = load_pop<STORE_FP32>(a, i, nbm.src(i), make_float2(0.0f, 0.0f));
                fr[i] = v.x;
                fb[i] = v.y;
            }
#pragma unroll
            for (int i = 0; i < 27; ++i) {
                const float s = fr[i] + fb[i];
                rho += s;
                if (cz(i) != 0) jz += (float)cz(i) * s;
            }
            const float Fz = (rho - a.rho_b0) * a.gz;
            const float lam_raw = (jz + 0.5f * Fz) / rho;
            const float lam = fminf(fmaxf(lam_raw, 0.0f), 1.0f);
            const float inv = 1.0f / (1.0f + lam);
            const float2 lrN = g.lr_out[(size_t)N * P + pxy];
            float lvr[27], lvb[27];
            float llam = 0.0f;
#pragma unroll
            for (int i = 0; i < 27; ++i) {
                const size_t hr = (size_t)i * P + pxy, hb = (size_t)(27 + i) * P + pxy;
                lvr[i] = g.lc[hr] + lrN.x + g.lh_in[hr];
                lvb[i] = g.lc[hb] + lrN.y + g.lh_in[hb];
                g.lh_out[hr] = lvr[i] * inv;
                g.lh_out[hb] = lvb[i] * inv;
                llam = fmaf(lvr[i], fr[i] - a.hist_out[hr], llam);
                llam = fmaf(lvb[i], fb[i] - a.hist_out[hb], llam);
            }
            llam *= inv;
            const bool active = lam_raw > 0.0f && lam_raw < 1.0f;
            const float inv_rho = 1.0f / rho;
#pragma unroll
            for (int i = 0; i < 27; ++i) {
                const float dl = active ? llam * ((float)cz(i) + 0.5f * a.gz - lam_raw) * inv_rho : 0.0f;
                float2 *slot = g.lp_out + (size_t)i * a.NN + nbm.src(i);
                float2 v = *slot;
                v.x += fmaf(lvr[i], lam * inv, dl);
                v.y += fmaf(lvb[i], lam * inv, dl);
                *slot = v;
            }
        }
    }
    block_accumulate<17>(part, g.acc_inlet, block_id());
}

// ------------------------------------------------------------------- objectives
// (phi, rho) of a post-collision state: rho_k = sum_i S_i^k.
__global__ void __launch_bounds__(256) obj_fields_kernel(StepArgs a, float2 *ph) {
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < a.NN; n += (long long)gridDim.x * blockDim.x) {
        float rr = 0.0f, rb = 0.0f;
#pragma unroll
        for (int i = 0; i < 27; ++i) {
            const float2 v = load_pop<STORE_FP32>(a, i, (int)n, make_float2(0.0f, 0.0f));
            rr += v.x;
            rb += v.y;
        }
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
static dim3 col_block() { return dim3(32, 8, 1); }
static dim3 col_grid(const StepArgs &a) { return dim3((a.nx + 31) / 32, (a.ny + 7) / 8, 1); }

long long adj_collide_blocks(const StepArgs &a) {
    const dim3 gr = node_grid(a);
    return (long long)gr.x * gr.y * gr.z;
}
long long adj_boundary_blocks(const StepArgs &a) {
    const dim3 gr = col_grid(a);
    return (long long)gr.x * gr.y * gr.z;
}

cudaError_t launch_adjoint_step(const StepArgs &a, const AdjArgs &g, cudaStream_t s, long long *launches) {
    const bool force = a.gx != 0.0f || a.gy != 0.0f || a.gz != 0.0f;
    if (force)
        adj_collide_kernel<true><<<node_grid(a), node_block(), 0, s>>>(a, g);
    else
        adj_collide_kernel<false><<<node_grid(a), node_block(), 0, s>>>(a, g);
    adj_stencil_kernel<<<node_grid(a), node_block(), 0, s>>>(a, g);
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
        adj_stencil_kernel<<<node_grid(a), node_block(), 0, s>>>(ao, o);
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
