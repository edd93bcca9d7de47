// lbcm_node.cuh -- per-node pieces shared by the forward step and its adjoint: the
// pull gather of the post-stream populations, the isotropic gradient stencil, the moments
// the paper-rate collision needs and the inverse 1-D central-moment sweep coefficients
// (arXiv:1804.08923, Section II).
#pragma once
#include "lbcm_device.cuh"

namespace lbcm {

// Direction i of the gather: the boundary planes at z = 0 / z = N, else the pull from the
// source node, reading the populations of direction j there.  With the fitted FP16 encoding
// the pull is loaded and decoded unconditionally (the source offsets are clamped onto the
// lattice, so the address is valid on the boundary planes too) and the boundary value replaces
// it afterwards: with the load inside the branch, the long decoding kept real branches around
// each load, which then could not be issued together (the phase-field pass ran 3x slower).
// The other storages keep the load inside the branch, which measured faster for them.
template <int S>
__device__ __forceinline__ void gather_one(const StepArgs &a, const Nbr &nb, int i, bool lo, bool slip_hi, size_t P,
                                           const Own &own, int j, float (&fr)[27], float (&fb)[27]) {
    if constexpr (S == STORE_FP16_FIT) {
        const float2 v = load_pop<S>(a, i, nb.src(i), own, j);
        fr[i] = v.x;
        fb[i] = v.y;
    }
    if (cz(i) == 1 && lo) {
        fr[i] = a.zin[zrank(i) * P + nb.pxy];
        fb[i] = a.zin[(9 + zrank(i)) * P + nb.pxy];
    } else if (cz(i) == -1 && slip_hi) {
        fr[i] = a.zout[zrank(i) * P + nb.pxy];
        fb[i] = a.zout[(9 + zrank(i)) * P + nb.pxy];
    } else if constexpr (S != STORE_FP16_FIT) {
        const float2 v = load_pop<S>(a, i, nb.src(i), own, j);
        fr[i] = v.x;
        fb[i] = v.y;
    }
}

// Post-stream populations of node (x, y, z) (Eq. (9), pull form) with the boundary
// planes of this step substituted.  Branches are uniform across a warp (one z per warp).
// kEdge = false: the caller knows that 0 < z < nz - 1, and the boundary-plane tests of every
// direction drop out of the code.
template <int S, bool W, bool kEdge = true>
__device__ __forceinline__ void gather(const StepArgs &a, const Nbr &nb, int z, float (&fr)[27], float (&fb)[27]) {
    const size_t P = (size_t)a.plane;
    const int N = a.nz - 1;
    const bool periodic_z = a.bc_zlo == BC_PERIODIC;
    const bool lo = kEdge && (z == 0) && !periodic_z;
    const bool conv = kEdge && (z == N) && a.bc_zhi == BC_CONVECTIVE;
    const bool slip_hi = kEdge && (z == N) && a.bc_zhi == BC_FREESLIP;
    if (conv) {
#pragma unroll
        for (int i = 0; i < 27; ++i) {
            fr[i] = a.hist_out[i * P + nb.pxy];
            fb[i] = a.hist_out[(27 + i) * P + nb.pxy];
        }
        return;
    }
    const Own own = reader_shift<S>(a, nb.n);
    // W: the lattice has side walls, where a pull reflects (the direction leaving the source is
    // nb.pulled(i), selected at run time).  Only warps holding a wall node take that path; the
    // others, and lattices without side walls, index every plane at compile time.
    bool reflect = false;
    if constexpr (W) reflect = __any_sync(__activemask(), nb.wxl || nb.wxh || nb.wyl || nb.wyh);
    if (reflect) {
        if constexpr (S == STORE_FP16_FIT) {
            const OwnFlip of = flip_own(own, nb.wxl, nb.wxh, nb.wyl, nb.wyh);
#pragma unroll
            for (int i = 0; i < 27; ++i) {
                const float2 v = load_pop_flip(a, i, nb.src(i), of, nb.pulled(i));
                fr[i] = v.x;
                fb[i] = v.y;
                if (cz(i) == 1 && lo) {
                    fr[i] = a.zin[zrank(i) * P + nb.pxy];
                    fb[i] = a.zin[(9 + zrank(i)) * P + nb.pxy];
                } else if (cz(i) == -1 && slip_hi) {
                    fr[i] = a.zout[zrank(i) * P + nb.pxy];
                    fb[i] = a.zout[(9 + zrank(i)) * P + nb.pxy];
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < 27; ++i) gather_one<S>(a, nb, i, lo, slip_hi, P, own, nb.pulled(i), fr, fb);
        }
    } else if constexpr (S == STORE_FP16_FIT) {
        // opposite pulls (i, i+1) were both encoded for this node, with odd terms of opposite
        // sign: one odd sum and one odd product decode the pair
        const float2 *rest = reinterpret_cast<const float2 *>(a.pin);
        const __half2 *mov = reinterpret_cast<const __half2 *>(rest + a.NN);
        const float2 f0 = __ldg(rest + nb.src(0));
        fr[0] = f0.x;
        fb[0] = f0.y;
#pragma unroll
        for (int i = 1; i < 27; i += 2) {
            const float2 hp = __half22float2(__ldg(mov + (size_t)(i - 1) * a.NN + nb.src(i)));
            const float2 hm = __half22float2(__ldg(mov + (size_t)i * a.NN + nb.src(i + 1)));
            const __half2 e = fit_odd_h(a, i, odd_sum(i, own));
            const float2 pp = fit_pred_h(a, i, own.Ah, e), pm = fit_pred_h(a, i, own.Ah, __hneg2(e));
            fr[i] = fmaf(hp.x, a.inv_dev_scale, pp.x);
            fb[i] = fmaf(hp.y, a.inv_dev_scale, pp.y);
            fr[i + 1] = fmaf(hm.x, a.inv_dev_scale, pm.x);
            fb[i + 1] = fmaf(hm.y, a.inv_dev_scale, pm.y);
        }
#pragma unroll
        for (int i = 1; i < 27; ++i) {
            if (cz(i) == 1 && lo) {
                fr[i] = a.zin[zrank(i) * P + nb.pxy];
                fb[i] = a.zin[(9 + zrank(i)) * P + nb.pxy];
            } else if (cz(i) == -1 && slip_hi) {
                fr[i] = a.zout[zrank(i) * P + nb.pxy];
                fb[i] = a.zout[(9 + zrank(i)) * P + nb.pxy];
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < 27; ++i) gather_one<S>(a, nb, i, lo, slip_hi, P, own, i, fr, fb);
    }
}

// Isotropic gradients of phi and rho (end of Section II): grad chi = 3 sum_j w_j chi(x + c_j)
// c_j, summed over the 13 pairs of opposite directions (j, j+1) as 3 w_j c_j (chi(x + c_j) -
// chi(x - c_j)), so that a uniform field gives exactly zero and nearby values subtract
// exactly.  Ghosts: z = -1 is phi = 1, rho = rho_r0 inside the inlet disc and the mirror of
// z = 0 elsewhere; z = N + 1 mirrors z = N.  kEdge = false: the caller knows that z > 0.
template <int S, bool kEdge = true>
__device__ __forceinline__ void stencil_gradients(const StepArgs &a, const Nbr &nb, int z, float &gpx, float &gpy,
                                                  float &gpz, float &grx, float &gry, float &grz) {
    const bool inlet_lo = kEdge && z == 0 && a.bc_zlo == BC_INLET;
    float ph[27], rh[27];
#pragma unroll
    for (int j = 1; j < 27; ++j) {
        // ghost planes were clamped onto z = 0 / z = N (mirror)
        if constexpr (S == STORE_FP32) {
            const float2 v = __ldg(a.phase + nb.nbr(j));
            ph[j] = v.x;
            rh[j] = v.y;
        } else if constexpr (S == STORE_FP16) {
            const float4 v = __ldg(a.ph_cur + nb.nbr(j));
            ph[j] = v.x;
            rh[j] = v.y;
        } else {
            const float4 v = __ldg(a.ph_cur + nb.nbr(j));
            ph[j] = v.x;
            rh[j] = fit_entry_rho(v);
        }
        if (cz(j) == -1 && inlet_lo) {
            if (a.disc[nb.yo[1 - cy(j)] + nb.xo[1 - cx(j)]]) {  // z = -1 inside the inlet disc
                ph[j] = 1.0f;
                rh[j] = a.rho_r0;
            }
        }
    }
    gpx = gpy = gpz = grx = gry = grz = 0.0f;
#pragma unroll
    for (int j = 1; j < 27; j += 2) {  // c_{j+1} = -c_j
        const float w3 = 3.0f * wgt(j);
        const float dp = ph[j] - ph[j + 1], dr = rh[j] - rh[j + 1];
        if (cx(j) != 0) { gpx = fmaf(w3 * cx(j), dp, gpx); grx = fmaf(w3 * cx(j), dr, grx); }
        if (cy(j) != 0) { gpy = fmaf(w3 * cy(j), dp, gpy); gry = fmaf(w3 * cy(j), dr, gry); }
        if (cz(j) != 0) { gpz = fmaf(w3 * cz(j), dp, gpz); grz = fmaf(w3 * cz(j), dr, grz); }
    }
}

// Coefficients of the inverse 1-D sweep: a value at c in {-1, 0, +1} from central moments
// (m0, m1, m2) about u is G0[c] m0 + G1[c] m1 + G2[c] m2 with
//   G0 = ((u^2 - u)/2, 1 - u^2, (u^2 + u)/2), G1 = (u - 1/2, -2u, u + 1/2), G2 = (1/2, -1, 1/2).
struct InvAxis {
    float g0[3], g1[3];
    __device__ __forceinline__ explicit InvAxis(float u) {
        const float u2 = u * u;
        g0[0] = 0.5f * (u2 - u);
        g0[1] = 1.0f - u2;
        g0[2] = 0.5f * (u2 + u);
        g1[0] = u - 0.5f;
        g1[1] = -2.0f * u;
        g1[2] = u + 0.5f;
    }
};
__device__ __forceinline__ constexpr float g2c(int c) { return c == 0 ? -1.0f : 0.5f; }

// Moments of the post-stream populations of one node that the paper-rate collision needs:
// colour densities, colour-blind mass, momentum and raw second moment.
struct Moments {
    float rho_r, rho_b, sf, jx, jy, jz, pxx, pyy, pzz, pxy, pxz, pyz;
};

// The moments above of gathered populations (fr, fb).  Every step kernel that needs them
// forms them here, in this one order, so that the moment pass and the adjoint's recompute
// see the same bits.
__device__ __forceinline__ void moments_of(const float (&fr)[27], const float (&fb)[27], Moments &m) {
    float sf, jx = 0.0f, jy = 0.0f, jz = 0.0f;
    float pxx = 0.0f, pyy = 0.0f, pzz = 0.0f, pxy = 0.0f, pxz = 0.0f, pyz = 0.0f;
    MassAcc mr, mb;  // the phase-field kernel's association
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        mr.add(i, fr[i]);
        mb.add(i, fb[i]);
    }
    // opposite pairs (i, i+1): odd moments take the difference, even ones the sum
    sf = fr[0] + fb[0];
#pragma unroll
    for (int i = 1; i < 27; i += 2) {
        const float fp = fr[i] + fb[i], fm = fr[i + 1] + fb[i + 1];
        const float s2 = fp + fm, d2 = fp - fm;
        sf += s2;
        if (cx(i) > 0) jx += d2; else if (cx(i) < 0) jx -= d2;
        if (cy(i) > 0) jy += d2; else if (cy(i) < 0) jy -= d2;
        if (cz(i) > 0) jz += d2; else if (cz(i) < 0) jz -= d2;
        if (cx(i) != 0) pxx += s2;
        if (cy(i) != 0) pyy += s2;
        if (cz(i) != 0) pzz += s2;
        if (cx(i) * cy(i) > 0) pxy += s2; else if (cx(i) * cy(i) < 0) pxy -= s2;
        if (cx(i) * cz(i) > 0) pxz += s2; else if (cx(i) * cz(i) < 0) pxz -= s2;
        if (cy(i) * cz(i) > 0) pyz += s2; else if (cy(i) * cz(i) < 0) pyz -= s2;
    }
    m = Moments{mr.total(), mb.total(), sf, jx, jy, jz, pxx, pyy, pzz, pxy, pxz, pyz};
}

// The collision moments of a node as the moment pass stores them: three float4 planes of NN
// entries, (rho_r, rho_b, sf, jx), (jy, jz, pxx, pyy), (pzz, pxy, pxz, pyz).
__device__ __forceinline__ void store_moments(float4 *__restrict__ mom, size_t NN, int n, const Moments &m) {
    mom[n] = make_float4(m.rho_r, m.rho_b, m.sf, m.jx);
    mom[NN + n] = make_float4(m.jy, m.jz, m.pxx, m.pyy);
    mom[2 * NN + n] = make_float4(m.pzz, m.pxy, m.pxz, m.pyz);
}
__device__ __forceinline__ Moments load_moments(const float4 *__restrict__ mom, size_t NN, int n) {
    const float4 a = __ldg(mom + n), b = __ldg(mom + NN + n), c = __ldg(mom + 2 * NN + n);
    return Moments{a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
}

// The same for the fused step kernel, where the moments were written earlier in the same launch
// and are read once: L1 is bypassed (ld.global.cg), and the L2 lines can be dropped afterwards.
__device__ __forceinline__ Moments load_moments_once(const float4 *__restrict__ mom, size_t NN, int n) {
    const float4 a = __ldcg(mom + n), b = __ldcg(mom + NN + n), c = __ldcg(mom + 2 * NN + n);
    return Moments{a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
}

// L2 cache policy that keeps lines over evict-first and evict-normal ones.
__device__ __forceinline__ unsigned long long l2_evict_last_policy() {
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void st_keep(float4 *p, float4 v, unsigned long long pol) {
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(v.x), "f"(v.y),
                 "f"(v.z), "f"(v.w), "l"(pol)
                 : "memory");
}
// Moments stored with the evict-last policy (the fused step kernel reads them a few planes later).
__device__ __forceinline__ void store_moments_keep(float4 *__restrict__ mom, size_t NN, int n, const Moments &m,
                                                   unsigned long long pol) {
    st_keep(mom + n, make_float4(m.rho_r, m.rho_b, m.sf, m.jx), pol);
    st_keep(mom + NN + n, make_float4(m.jy, m.jz, m.pxx, m.pyy), pol);
    st_keep(mom + 2 * NN + n, make_float4(m.pzz, m.pxy, m.pxz, m.pyz), pol);
}
// Drops the 128-byte L2 line at p (128-byte aligned) without writing it back: its contents
// become undefined.  For data that is dead (read for the last time by every thread that
// shares the line).
__device__ __forceinline__ void l2_discard(const void *p) {
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}

}  // namespace lbcm
