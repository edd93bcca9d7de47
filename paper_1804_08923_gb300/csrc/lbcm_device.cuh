// lbcm_device.cuh -- D3Q27 lattice constants and per-node device math of the
// colour-gradient central-moment LB step (arXiv:1804.08923, Section II), FP32.
//
// Everything here is compile-time unrolled over the 27 directions so that direction
// indices fold into immediates and the 27-vectors live in registers.
#pragma once
#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

namespace lbcm {

// Velocity set of Eq. (8): c+1 packed two bits per direction.
constexpr unsigned long long kPackX = 0x20888895489549ull;
constexpr unsigned long long kPackY = 0x0a089548a09495ull;
constexpr unsigned long long kPackZ = 0x08a0a0a0954955ull;

__host__ __device__ constexpr int cx(int i) { return (int)((kPackX >> (2 * i)) & 3ull) - 1; }
__host__ __device__ constexpr int cy(int i) { return (int)((kPackY >> (2 * i)) & 3ull) - 1; }
__host__ __device__ constexpr int cz(int i) { return (int)((kPackZ >> (2 * i)) & 3ull) - 1; }
__host__ __device__ constexpr int csq(int i) { return cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i); }
// position of direction i in the 3x3x3 tensor-product array [cx+1][cy+1][cz+1]
__host__ __device__ constexpr int cell(int i) { return (cx(i) + 1) * 9 + (cy(i) + 1) * 3 + (cz(i) + 1); }
// Inverse maps as packed tables built at compile time, so that a call with a run-time
// argument (a direction reflected at a side wall at run time) is a shift and a mask, not a loop.
__host__ __device__ constexpr int dir_search(int x, int y, int z) {
    int r = 0;
    for (int j = 0; j < 27; ++j)
        if (cx(j) == x && cy(j) == y && cz(j) == z) r = j;
    return r;
}
// 5-bit direction index of cell (x+1)*9 + (y+1)*3 + (z+1), 12 cells per word
__host__ __device__ constexpr unsigned long long pack_dirs(int word) {
    unsigned long long w = 0;
    for (int k = 0; k < 12; ++k) {
        const int c = word * 12 + k;
        if (c < 27) w |= (unsigned long long)dir_search(c / 9 - 1, (c / 3) % 3 - 1, c % 3 - 1) << (5 * k);
    }
    return w;
}
constexpr unsigned long long kDirOf0 = pack_dirs(0), kDirOf1 = pack_dirs(1), kDirOf2 = pack_dirs(2);
// direction with velocity (x, y, z)
__host__ __device__ constexpr int dir_of(int x, int y, int z) {
    const int c = (x + 1) * 9 + (y + 1) * 3 + (z + 1);
    const unsigned long long w = c < 12 ? kDirOf0 : (c < 24 ? kDirOf1 : kDirOf2);
    return (int)((w >> (5 * (c % 12))) & 31ull);
}
// direction with c_z flipped (specular reflection on a z wall)
__host__ __device__ constexpr int mirror_z(int i) { return dir_of(cx(i), cy(i), -cz(i)); }
// direction i with c_x, c_y or both reversed (specular reflection on a side wall)
__host__ __device__ constexpr int flip_x(int i) { return dir_of(-cx(i), cy(i), cz(i)); }
__host__ __device__ constexpr int flip_y(int i) { return dir_of(cx(i), -cy(i), cz(i)); }
__host__ __device__ constexpr int flip_xy(int i) { return dir_of(-cx(i), -cy(i), cz(i)); }
// rank of direction i among those with the same c_z = +1 (or -1), 0..8; 4 bits per direction
__host__ __device__ constexpr int zrank_search(int i) {
    int r = 0;
    for (int j = 0; j < i; ++j)
        if (cz(j) == cz(i)) ++r;
    return r;
}
__host__ __device__ constexpr unsigned long long pack_zrank(int word) {
    unsigned long long w = 0;
    for (int k = 0; k < 16; ++k)
        if (word * 16 + k < 27) w |= (unsigned long long)zrank_search(word * 16 + k) << (4 * k);
    return w;
}
constexpr unsigned long long kZrank0 = pack_zrank(0), kZrank1 = pack_zrank(1);
__host__ __device__ constexpr int zrank(int i) {
    return (int)(((i < 16 ? kZrank0 : kZrank1) >> (4 * (i & 15))) & 15ull);
}
// the tables against the searches they replace
constexpr bool check_tables() {
    for (int i = 0; i < 27; ++i) {
        if (dir_of(cx(i), cy(i), cz(i)) != i || zrank(i) != zrank_search(i)) return false;
        if (cz(mirror_z(i)) != -cz(i) || cx(flip_x(i)) != -cx(i) || cy(flip_y(i)) != -cy(i)) return false;
    }
    return true;
}
static_assert(check_tables(), "direction tables");

// D3Q27 weights
__host__ __device__ constexpr float wgt(int i) {
    return csq(i) == 0 ? 8.0f / 27.0f : csq(i) == 1 ? 2.0f / 27.0f : csq(i) == 2 ? 1.0f / 54.0f : 1.0f / 216.0f;
}
// Eq. (31)
__host__ __device__ constexpr float bcoef(int i) {
    return csq(i) == 0 ? -10.0f / 27.0f : wgt(i);
}
// Eq. (20): varphi_i(alpha) = alpha (rest) or k_q (1 - alpha)
__host__ __device__ constexpr float varphi_k(int i) {
    return csq(i) == 1 ? 2.0f / 19.0f : csq(i) == 2 ? 1.0f / 38.0f : 1.0f / 152.0f;
}
__device__ __forceinline__ float varphi(int i, float alpha, float one_m_alpha) {
    return csq(i) == 0 ? alpha : varphi_k(i) * one_m_alpha;
}
// Eq. (21): coefficient of nu (G : c c) by speed class, G : c c = (c.u)(c.grad rho)/24
__host__ __device__ constexpr float phi_corr(int i) {
    return csq(i) == 1 ? 16.0f / 24.0f : csq(i) == 2 ? 4.0f / 24.0f : 1.0f / 24.0f;
}
// 1/|c_i| for the recolouring angle (0 for the rest direction)
__host__ __device__ constexpr float inv_cnorm(int i) {
    return csq(i) == 0 ? 0.0f : csq(i) == 1 ? 1.0f : csq(i) == 2 ? 0.70710678118654752f : 0.57735026918962576f;
}

// Polynomial part of Eq. (18): 3 cu + 9/2 cu^2 - 3/2 u^2 + 9/2 cu^3 - 9/2 cu u^2
__device__ __forceinline__ float eq_poly(float cu, float usq) {
    float t = fmaf(4.5f, cu, 3.0f);            // 3 + 4.5 cu
    t = fmaf(4.5f * cu, cu, t) - 4.5f * usq;  // 3 + 4.5cu + 4.5cu^2 - 4.5u^2
    return fmaf(cu, t, -1.5f * usq);          // cu * (...) - 1.5 u^2
}

// SplitMix64 (Steele, Lea and Flood 2014): gamma increment and finaliser.
__host__ __device__ __forceinline__ unsigned long long splitmix64(unsigned long long s) {
    unsigned long long z = s + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
// Inlet noise xi in [-1, 1) for (seed, step, x, y): top 24 bits of a double hash, exact.
__host__ __device__ __forceinline__ float inlet_xi(unsigned long long seed, long long step, int x, int y, int nx, int ny) {
    unsigned long long idx = ((unsigned long long)step * (unsigned long long)ny + (unsigned long long)y) *
                                 (unsigned long long)nx + (unsigned long long)x;
    unsigned long long h = splitmix64(seed ^ splitmix64(idx));
    return (float)(unsigned int)(h >> 40) * (1.0f / 8388608.0f) - 1.0f;
}

// Inlet velocity at source column (xs, ys) of the disc: plug u_in times the Fourier profile
// 1 + sum_m (a_m cos m theta + b_m sin m theta) along z, plus the radial noise a u_in xi rhat.
// cos m theta, sin m theta come from the angle-addition recurrence on the unit offset.
struct InletVel {
    float ux, uy, uz;
    float dux, duy, prof;  // d(ux, uy, uz)/d u_in = (dux, duy, prof)
    float cm[9], sm[9];    // cos m theta, sin m theta for m = 0..8
};

__device__ __forceinline__ void inlet_velocity(float u_in, float noise_amp, const float *fourier, float xc, float yc,
                                               unsigned long long seed, long long step, int xs, int ys, int nx, int ny,
                                               InletVel &v) {
    const float rx = (float)xs - xc, ry = (float)ys - yc;
    const float r = sqrtf(rx * rx + ry * ry);
    const float c1 = r > 0.0f ? rx / r : 1.0f, s1 = r > 0.0f ? ry / r : 0.0f;
    const float unit = noise_amp * inlet_xi(seed, step, xs, ys, nx, ny);
    const float amp = unit * u_in;
    v.ux = r > 0.0f ? amp * rx / r : 0.0f;
    v.uy = r > 0.0f ? amp * ry / r : 0.0f;
    v.dux = r > 0.0f ? unit * rx / r : 0.0f;
    v.duy = r > 0.0f ? unit * ry / r : 0.0f;
    v.cm[0] = 1.0f;
    v.sm[0] = 0.0f;
    float prof = 1.0f;
#pragma unroll
    for (int m = 1; m <= 8; ++m) {
        v.cm[m] = v.cm[m - 1] * c1 - v.sm[m - 1] * s1;
        v.sm[m] = v.sm[m - 1] * c1 + v.cm[m - 1] * s1;
        prof = fmaf(fourier[2 * (m - 1)], v.cm[m], fmaf(fourier[2 * m - 1], v.sm[m], prof));
    }
    v.prof = prof;
    v.uz = u_in * prof;
}

// 1 - alpha-bar (Eq. (27) as printed, (1 + phi)/2 alpha_r + (1 - phi)/2 alpha_b, or by mass
// fractions), formed from the colours' 1 - alpha_k (oma_r, oma_b, rounded once from FP64): at
// large density ratios alpha-bar is close to 1 and 1 - alpha-bar computed by subtraction in
// FP32 would keep only a few significant digits of the moving equilibrium populations and of
// the equation of state (Eq. (26)).
__device__ __forceinline__ float one_minus_alpha_bar(int mix, float rho_r, float rho_b, float inv_rho, float hp,
                                                     float hm, float oma_r, float oma_b) {
    return mix ? (rho_r * oma_r + rho_b * oma_b) * inv_rho : hp * oma_r + hm * oma_b;
}

// Sum of one colour's 27 populations of a node in one fixed association,
//   f_0 + (((f_1 + f_2) + (f_3 + f_4)) + ... + (f_25 + f_26)),
// the one the collision uses when it writes the rest population as the remainder rho_k - s of
// the moving ones.  A reader that gathers the same moving values therefore gets rho_k back
// (fl(fl(rho - s) + s) = rho up to a rounding tie), so a uniform state is an exact fixed point
// of the FP32 step instead of drifting by an ulp of density now and then; a drift that, being
// the same at every node, would not average out and, against the frozen convective plane,
// would drive a spurious outflow velocity.  add(i, v) must be called in the order i = 0..26
// (or 1..26 for the moving part s alone).
struct MassAcc {
    float f0 = 0.0f, odd = 0.0f, s = 0.0f;
    __device__ __forceinline__ void add(int i, float v) {
        if (i == 0)
            f0 = v;
        else if (i & 1)
            odd = v;
        else
            s += odd + v;
    }
    __device__ __forceinline__ float total() const { return f0 + s; }
};

// Order parameter of Eq. (23) from the colour densities (1/rho_k0 given).
__device__ __forceinline__ float order_parameter(float rho_r, float rho_b, float inv_rho_r0, float inv_rho_b0) {
    const float A = rho_r * inv_rho_r0, B = rho_b * inv_rho_b0;
    return (A - B) / (A + B);
}

enum { BC_PERIODIC = 0, BC_FREESLIP = 1, BC_INLET = 2, BC_CONVECTIVE = 3 };

// Population storage.  FP32: float2 pop[27][NN], (red, blue) of direction i at node n.
// FP16: float2 rest[NN] (direction 0, FP32) followed by __half2 mov[26][NN] holding, for
// i >= 1, h_i^k = f_i^k - rho_k(d) varphi_i(alpha_k): the deviation from the rest
// equilibrium of the node d = y + c_i that will read it (pull streaming), so that a node
// decodes everything it gathers with its own colour densities.  Those come from a float4
// (phi, rho, rho_r, rho_b) phase buffer that pairs with each population buffer.
// FP16_FIT: the same layout, with h_i^k = S_h (f_i^k - P_i^k(d)) against a per-reader
// prediction P_i^k = A_k k_q(i) + w_i c_i . v_k / S_v.  A_k = rho_k (1 - alpha-bar) is the even
// (rest-equilibrium) part with the mixture's alpha-bar; v_k, the odd part, is the least-squares
// fit sum_i (f_i^k - w_i c_i . v)^2 -> min over the 26 moving populations the reader gathered
// in the step before (v_k = 72 sum_i w_i c_i f_i^k, since sum_i w_i^2 c_ix^2 = 1/72), stored
// as FP8 e4m3 scaled by the power of two S_v.  The phase entry packs it all into 16 bytes
// (pack_fit_entry): phi (FP32), (A_r, A_b) as half2, the six FP8 values and rho in half
// precision (rho enters only the gradient of the Phi correction); S_h is a power of two that
// lifts the deviations out of the FP16 subnormal range.  Near an interface the recolouring and the reader-writer density
// difference make h large under the rest shift; the fitted prediction removes most of it.
enum { STORE_FP32 = 0, STORE_FP16 = 1, STORE_FP16_FIT = 2 };

// Everything a step kernel needs, passed by value.
struct StepArgs {
    const void *__restrict__ pin;       // S(t)
    void *__restrict__ pout;            // S(t+1)
    float2 *__restrict__ phase;         // FP32 storage: post-stream (phi, rho) of step t+1
    const float4 *__restrict__ ph_prev; // FP16: (phi, rho, rho_r, rho_b) that S(t) was encoded with
    float4 *__restrict__ ph_cur;        // FP16: post-stream (phi, rho, rho_r, rho_b) of step t+1
                                        // (FP16_FIT: the packed entry of pack_fit_entry)
    float4 *__restrict__ mom;           // collision moments of step t+1, written by the moment pass
                                        // and read by the collision: [3][NN] float4
    const float *__restrict__ hist_in;  // outflow plane f(N, t): [2][27][ny][nx]
    float *__restrict__ hist_out;       // outflow plane f(N, t+1)
    float *__restrict__ zin;            // incoming z=0 populations (c_z = +1): [2][9][ny][nx]
    float *__restrict__ zout;           // incoming z=N populations (c_z = -1) on a free-slip top
    const uint8_t *__restrict__ disc;   // inlet disc membership [ny][nx]
    long long NN, plane;                // nodes, nx*ny
    int nx, ny, nz, bc_zlo, bc_zhi;
    int wall_x, wall_y;                 // free-slip side walls (else periodic)
    int alpha_mix;                      // alpha-bar by (1 +- phi)/2 (0) or by mass fraction (1)
    float rho_r0, rho_b0, inv_rho_r0, inv_rho_b0;
    float alpha_r, alpha_b, inv_nu_r, inv_nu_b;
    float oma_r, oma_b;                 // 1 - alpha_r, 1 - alpha_b (rounded once from FP64)
    float sigma, beta, eps2;
    float gx, gy, gz;
    float s0, s1, s2b, s3, s4, s5, s6;
    float u_in, noise_amp, xc, yc;
    float shift_r[4], shift_b[4];       // varphi_i(alpha_k) by speed class |c|^2 = 1..3 (FP16 shift)
    float wv[4];                        // FP16_FIT: w_q / S_v by speed class
    __half2 kqh[4], wvh[4];             // FP16_FIT prediction: k_q and w_q / S_v in half precision
    float dev_scale, inv_dev_scale;     // FP16_FIT: S_h, 1/S_h (powers of two)
    float v_scale;                      // FP16_FIT: S_v (power of two)
    float fourier[16];                  // inlet profile coefficients a_1, b_1, ..., a_8, b_8
    // optional outputs for the adjoint's recompute (NULL otherwise): the gradients of every
    // node, grad4[NN] = (gpx, gpy, gpz, grx) and grad2[NN] = (gry, grz) (with the moments the
    // moment pass writes to mom, the collision's inputs); fm_out[2][27][nx ny] = f(N-1, t+1) of
    // the outflow columns
    float4 *__restrict__ grad4;
    float2 *__restrict__ grad2;
    float *__restrict__ fm_out;
    unsigned long long seed;
    long long step;  // index of the step being taken (state t -> t+1 uses t)
    int z_base;      // first plane of the launch (a launch covers planes z_base .. z_base + gridDim.z - 1)
};

// Shift weight varphi_i(alpha_k) of the FP16 encoding (same value at encode and decode).
__device__ __forceinline__ float2 shift_w(const StepArgs &a, int i) {
    return make_float2(a.shift_r[csq(i)], a.shift_b[csq(i)]);
}

// What a reading node decodes its incoming populations with: FP16, A = (rho_r, rho_b);
// FP16_FIT, A = (A_r, A_b) and v[d] = (v_r, v_b) along axis d, times S_v, widened from FP8 to
// half precision (exactly).  Unused for FP32.
struct Own {
    float2 A;      // FP16
    __half2 Ah;    // FP16_FIT
    __half2 v[3];  // FP16_FIT
};

__device__ __forceinline__ __half2 fp8x2_to_half2(unsigned int bits) {
    const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(bits & 0xffffu), __NV_E4M3);
    return __half2(h);
}

// FP16_FIT phase entry, bit fields of a float4: x = phi (FP32); y = (A_r, A_b) as half2;
// z = FP8 pairs (v_x | v_y << 16); w = FP8 pair v_z | half(rho) << 16.
__device__ __forceinline__ float4 pack_fit_entry(float phi, float rho, float2 A, uint2 q) {
    const __half2 Ah = __floats2half2_rn(A.x, A.y);
    const unsigned int rh = (unsigned int)__half_as_ushort(__float2half_rn(rho));
    return make_float4(phi, __uint_as_float(*reinterpret_cast<const unsigned int *>(&Ah)), __uint_as_float(q.x),
                       __uint_as_float((q.y & 0xffffu) | (rh << 16)));
}
__device__ __forceinline__ float fit_entry_rho(float4 e) {
    return __half2float(__ushort_as_half((unsigned short)(__float_as_uint(e.w) >> 16)));
}

template <int S>
__device__ __forceinline__ Own own_of(const float4 *ph, int n) {
    Own o{};
    if constexpr (S == STORE_FP16) {
        const float4 v = __ldg(ph + n);
        o.A = make_float2(v.z, v.w);
    } else if constexpr (S == STORE_FP16_FIT) {
        const float4 v = __ldg(ph + n);
        const unsigned int y = __float_as_uint(v.y), z = __float_as_uint(v.z), w = __float_as_uint(v.w);
        o.Ah = *reinterpret_cast<const __half2 *>(&y);
        o.v[0] = fp8x2_to_half2(z);
        o.v[1] = fp8x2_to_half2(z >> 16);
        o.v[2] = fp8x2_to_half2(w);
    }
    return o;
}

// FP16_FIT prediction P^k for the slot of direction j (class q of i = class of j), in half-precision
// arithmetic on both colours at once:
//   P = fl16(A k_q + fl16(w_q/S_v (c_j . v)))   (one HMUL2, one HFMA2; A, v, k_q, w_q/S_v in half)
// then widened to FP32.  One fixed sequence of operations, so that the writer and the reader get
// the same bits; a prediction needs no more precision than this (the deviation from it is what
// is stored, and the FP8 fit v is far coarser).  Opposite slots get exactly opposite odd terms
// (negation commutes with rounding to nearest), which lets a reader decode a pair of opposite
// pulls with one odd sum and one product (gather, lbcm_node.cuh).
__device__ __forceinline__ __half2 odd_sum(int j, const Own &o) {
    __half2 dh = __float2half2_rn(0.0f);
    if (cx(j) > 0) dh = __hadd2(dh, o.v[0]); else if (cx(j) < 0) dh = __hsub2(dh, o.v[0]);
    if (cy(j) > 0) dh = __hadd2(dh, o.v[1]); else if (cy(j) < 0) dh = __hsub2(dh, o.v[1]);
    if (cz(j) > 0) dh = __hadd2(dh, o.v[2]); else if (cz(j) < 0) dh = __hsub2(dh, o.v[2]);
    return dh;
}
// the odd term fl16(w_q/S_v (c_j . v)) of class q of i from the odd sum dh
__device__ __forceinline__ __half2 fit_odd_h(const StepArgs &a, int i, __half2 dh) {
    return __hmul2(a.wvh[csq(i)], dh);
}
// P from A and the odd term e
__device__ __forceinline__ float2 fit_pred_h(const StepArgs &a, int i, __half2 Ah, __half2 e) {
    return __half22float2(__hfma2(Ah, a.kqh[csq(i)], e));
}
__device__ __forceinline__ float2 fit_pred(const StepArgs &a, int i, int j, const Own &o) {
    return fit_pred_h(a, i, o.Ah, fit_odd_h(a, i, odd_sum(j, o)));
}

// Populations (red, blue) of direction j stored at node src, decoded to FP32; for FP16,
// own holds what the reading node, the node the value was encoded for, decodes with.  i is a
// direction with |c_i| = |c_j| (j itself, or the direction j is reflected from at a side wall):
// it selects the shift weight, so that an unrolled caller indexes the weights at compile time.
template <int S>
__device__ __forceinline__ float2 load_pop(const StepArgs &a, int i, int src, const Own &own, int j) {
    if constexpr (S == STORE_FP32) {
        return __ldg(reinterpret_cast<const float2 *>(a.pin) + (size_t)j * a.NN + src);
    } else {
        const float2 *rest = reinterpret_cast<const float2 *>(a.pin);
        if (i == 0) return __ldg(rest + src);
        const __half2 *mov = reinterpret_cast<const __half2 *>(rest + a.NN);
        const float2 h = __half22float2(__ldg(mov + (size_t)(j - 1) * a.NN + src));
        if constexpr (S == STORE_FP16) {
            const float2 w = shift_w(a, i);
            return make_float2(fmaf(own.A.x, w.x, h.x), fmaf(own.A.y, w.y, h.y));
        } else {
            const float2 p = fit_pred(a, i, j, own);
            return make_float2(fmaf(h.x, a.inv_dev_scale, p.x), fmaf(h.y, a.inv_dev_scale, p.y));
        }
    }
}
template <int S>
__device__ __forceinline__ float2 load_pop(const StepArgs &a, int i, int src, const Own &own) {
    return load_pop<S>(a, i, src, own, i);
}

// FP16_FIT decoding of pulls reflected at side walls.  The slot read is j = i with the
// crossing velocity components reversed; instead of evaluating c_j . v with a run-time j, the
// node negates its odd fit once per side (xp: components of directions with c_x > 0, xn: c_x <
// 0, likewise y), so the sum runs over compile-time signs of i.  The sums equal those of
// fit_pred for slot j bit for bit: 0 + (-v) = 0 - v and d + (-v) = d - v exactly.
struct OwnFlip {
    __half2 Ah;
    __half2 xp, xn, yp, yn, z;
};
__device__ __forceinline__ OwnFlip flip_own(const Own &o, bool wxl, bool wxh, bool wyl, bool wyh) {
    OwnFlip f;
    f.Ah = o.Ah;
    f.xp = wxl ? __hneg2(o.v[0]) : o.v[0];
    f.xn = wxh ? __hneg2(o.v[0]) : o.v[0];
    f.yp = wyl ? __hneg2(o.v[1]) : o.v[1];
    f.yn = wyh ? __hneg2(o.v[1]) : o.v[1];
    f.z = o.v[2];
    return f;
}
__device__ __forceinline__ float2 load_pop_flip(const StepArgs &a, int i, int src, const OwnFlip &o, int j) {
    const float2 *rest = reinterpret_cast<const float2 *>(a.pin);
    if (i == 0) return __ldg(rest + src);
    const __half2 *mov = reinterpret_cast<const __half2 *>(rest + a.NN);
    const float2 h = __half22float2(__ldg(mov + (size_t)(j - 1) * a.NN + src));
    __half2 dh = __float2half2_rn(0.0f);
    if (cx(i) > 0) dh = __hadd2(dh, o.xp); else if (cx(i) < 0) dh = __hsub2(dh, o.xn);
    if (cy(i) > 0) dh = __hadd2(dh, o.yp); else if (cy(i) < 0) dh = __hsub2(dh, o.yn);
    if (cz(i) > 0) dh = __hadd2(dh, o.z); else if (cz(i) < 0) dh = __hsub2(dh, o.z);
    const float2 p = fit_pred_h(a, i, o.Ah, fit_odd_h(a, i, dh));
    return make_float2(fmaf(h.x, a.inv_dev_scale, p.x), fmaf(h.y, a.inv_dev_scale, p.y));
}

// What node n decodes its gathered populations with (the entries S(t) was encoded for).
template <int S>
__device__ __forceinline__ Own reader_shift(const StepArgs &a, int n) {
    return own_of<S>(a.ph_prev, n);
}

// Store populations f of direction i at node n; dest = what the node n + c_i that will read
// them decodes with (FP16).  Returns the values that node will decode, so the caller can
// account for the storage rounding.
template <int S>
__device__ __forceinline__ float2 store_pop(const StepArgs &a, int i, int n, float2 f, const Own &dest) {
    if constexpr (S == STORE_FP32) {
        reinterpret_cast<float2 *>(a.pout)[(size_t)i * a.NN + n] = f;
        return f;
    } else {
        float2 *rest = reinterpret_cast<float2 *>(a.pout);
        if (i == 0) {
            rest[n] = f;
            return f;
        }
        __half2 *slot = reinterpret_cast<__half2 *>(rest + a.NN) + (size_t)(i - 1) * a.NN + n;
        if constexpr (S == STORE_FP16) {
            const float2 w = shift_w(a, i);
            const __half2 h = __floats2half2_rn(fmaf(-dest.A.x, w.x, f.x), fmaf(-dest.A.y, w.y, f.y));
            *slot = h;
            const float2 hf = __half22float2(h);
            return make_float2(fmaf(dest.A.x, w.x, hf.x), fmaf(dest.A.y, w.y, hf.y));
        } else {
            const float2 p = fit_pred(a, i, i, dest);
            const __half2 h = __floats2half2_rn((f.x - p.x) * a.dev_scale, (f.y - p.y) * a.dev_scale);
            *slot = h;
            const float2 hf = __half22float2(h);
            return make_float2(fmaf(hf.x, a.inv_dev_scale, p.x), fmaf(hf.y, a.inv_dev_scale, p.y));
        }
    }
}
__device__ __forceinline__ Own no_shift() { return Own{}; }

// FP16_FIT odd fit of the gathered populations, times S_v, as FP8 e4m3 pairs (red, blue) per
// axis: .x = x | y << 16, .y = z.
__device__ __forceinline__ uint2 fit_odd_fp8(const StepArgs &a, const float (&fr)[27], const float (&fb)[27]) {
    float vr[3] = {0.0f, 0.0f, 0.0f}, vb[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int i = 1; i < 27; i += 2) {  // c_{i+1} = -c_i: the pair contributes w_i c_i (f_i - f_{i+1})
        const float dr = wgt(i) * (fr[i] - fr[i + 1]), db = wgt(i) * (fb[i] - fb[i + 1]);
        if (cx(i) > 0) { vr[0] += dr; vb[0] += db; } else if (cx(i) < 0) { vr[0] -= dr; vb[0] -= db; }
        if (cy(i) > 0) { vr[1] += dr; vb[1] += db; } else if (cy(i) < 0) { vr[1] -= dr; vb[1] -= db; }
        if (cz(i) > 0) { vr[2] += dr; vb[2] += db; } else if (cz(i) < 0) { vr[2] -= dr; vb[2] -= db; }
    }
    const float sc = 72.0f * a.v_scale;
    unsigned int q[3];
#pragma unroll
    for (int d = 0; d < 3; ++d)
        q[d] = (unsigned int)__nv_cvt_float2_to_fp8x2(make_float2(vr[d] * sc, vb[d] * sc), __NV_SATFINITE, __NV_E4M3);
    return make_uint2(q[0] | (q[1] << 16), q[2]);
}

// FP16_FIT even part A_k = rho_k (1 - alpha-bar) of a node with colour densities (rr, rb) and
// order parameter phi (either reading of alpha-bar; one division only for the mass fraction).
__device__ __forceinline__ float2 fit_even(const StepArgs &a, float rr, float rb, float phi) {
    float oma;
    if (a.alpha_mix)
        oma = (rr * a.oma_r + rb * a.oma_b) / (rr + rb);
    else
        oma = 0.5f * (1.0f + phi) * a.oma_r + 0.5f * (1.0f - phi) * a.oma_b;
    return make_float2(rr * oma, rb * oma);
}

__device__ __forceinline__ int wrapi(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// 32-bit offsets of the node and of its three neighbouring columns, rows and planes:
// xo[d+1] = x - d, yo[d+1] = (y - d) nx, zo[d+1] = (z - d) nx ny for d = -1, 0, 1, wrapped
// where periodic and clamped onto the wall layer at walls (the half-way reflection returns to
// the node's own layer; gradient ghosts mirror it).  The pull
// source of direction i is zo[cz+1] + yo[cy+1] + xo[cx+1]; the neighbour x + c_j is
// zo[1-cz] + yo[1-cy] + xo[1-cx].  nx ny nz < 2^31 keeps every offset in 32 bits.
struct Nbr {
    int xo[3], yo[3], zo[3];
    int n, pxy;
    bool wxl, wxh, wyl, wyh;  // the node lies on a free-slip side wall (x = 0, x = nx-1, y = 0, y = ny-1)
    __device__ __forceinline__ Nbr(const StepArgs &a, int x, int y, int z) {
        const bool periodic_z = a.bc_zlo == BC_PERIODIC;
        const int N = a.nz - 1, P = (int)a.plane;
#pragma unroll
        for (int d = -1; d <= 1; ++d) {
            int zs = z - d;
            if (periodic_z) zs = wrapi(zs, a.nz);
            zs = min(max(zs, 0), N);
            zo[d + 1] = zs * P;
            const int ys = a.wall_y ? min(max(y - d, 0), a.ny - 1) : wrapi(y - d, a.ny);
            const int xs = a.wall_x ? min(max(x - d, 0), a.nx - 1) : wrapi(x - d, a.nx);
            yo[d + 1] = ys * a.nx;
            xo[d + 1] = xs;
        }
        pxy = yo[1] + x;
        n = zo[1] + pxy;
        wxl = a.wall_x && x == 0;
        wxh = a.wall_x && x == a.nx - 1;
        wyl = a.wall_y && y == 0;
        wyh = a.wall_y && y == a.ny - 1;
    }
    __device__ __forceinline__ int src(int i) const { return zo[cz(i) + 1] + yo[cy(i) + 1] + xo[cx(i) + 1]; }
    __device__ __forceinline__ int nbr(int j) const { return zo[1 - cz(j)] + yo[1 - cy(j)] + xo[1 - cx(j)]; }
    // whether the pull of direction i (source x - c_i) crosses a side wall in x / in y
    __device__ __forceinline__ bool fx(int i) const { return cx(i) > 0 ? wxl : (cx(i) < 0 ? wxh : false); }
    __device__ __forceinline__ bool fy(int i) const { return cy(i) > 0 ? wyl : (cy(i) < 0 ? wyh : false); }
    // the direction that leaves the (reflected) source of the pull of direction i
    __device__ __forceinline__ int pulled(int i) const {
        const bool bx = fx(i), by = fy(i);
        return bx ? (by ? flip_xy(i) : flip_x(i)) : (by ? flip_y(i) : i);
    }
    // whether the neighbour x + c_j lies beyond a side wall in x / in y (mirror ghost)
    __device__ __forceinline__ bool gx(int j) const { return cx(j) < 0 ? wxl : (cx(j) > 0 ? wxh : false); }
    __device__ __forceinline__ bool gy(int j) const { return cy(j) < 0 ? wyl : (cy(j) > 0 ? wyh : false); }
};

// What the node that will read direction i from node nb.n decodes with (FP16 encodings).
template <int S>
__device__ __forceinline__ Own dest_shift(const StepArgs &a, const Nbr &nb, int i) {
    return own_of<S>(a.ph_cur, nb.nbr(i));
}

// Populations (red, blue) of direction i stored at node nb.n, decoded (for FP16 with what
// the node that reads them decodes with; a.ph_cur must pair with a.pin).
template <int S>
__device__ __forceinline__ float2 stored_pop(const StepArgs &a, const Nbr &nb, int i) {
    return load_pop<S>(a, i, nb.n, dest_shift<S>(a, nb, i));
}

}  // namespace lbcm
