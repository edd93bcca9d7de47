// lbcm_step.cu -- the per-time-step kernels of the colour-gradient central-moment LB
// method (arXiv:1804.08923), FP32 populations and arithmetic, sm_103a.
//
// One step (state S(t) -> S(t+1)) is three launches on the context's stream:
//   1. boundary_plane_kernel  incoming z = 0 populations (inlet disc / free-slip mirror),
//                             free-slip top, and the convective outflow plane
//                             f(N, t+1) = [f(N, t) + lambda f(N-1, t+1)] / (1 + lambda)
//                             (Section IV.A).  One warp per (x, y) column.
//   2. moment_kernel          pull-gathers the 54 post-stream populations of a node (the
//                             step's only gather) and writes its order parameter phi
//                             (Eq. (23)) and total density rho (Section II, densities) for
//                             the gradient stencil, and the 12 moments the collision needs
//                             (colour densities, mass, momentum, raw second moment).  One
//                             thread per node.
//   3. collide_kernel         reads a node's moments, takes the isotropic gradients of phi
//                             and rho from the fields of step 2 (end of Section II), and
//                             applies the central-moment collision with the enhanced
//                             equilibrium and GMRT forcing (Eqs. (11), (18), (21), (28),
//                             (29)), the perturbation (Eq. (30)) and the recolouring
//                             (Eqs. (33), (34)); writes the 54 post-collision populations
//                             of the node (pull scheme: streaming happens in the next
//                             step's gathers).
// With relaxation rates other than the paper's, step 2 is phase_field_kernel (phase entry
// only) and step 3 collide_general_kernel, which gathers the populations again.
//
// The collision applies T^-1 K T through the tensor-product central moments
//   kappa_abc = sum_i f_i (c_ix - u_x)^a (c_iy - u_y)^b (c_iz - u_z)^c,  a, b, c in {0,1,2},
// computed by three 1-D shifted sweeps and undone by three reverse sweeps.  The 27 rows
// of the paper's moment set (Eq. (14)) are, order by order, invertible combinations
// of these; K holds one rate per order except order 2, where the trace relaxes with s_2b
// and the deviatoric part with s_2nu.  Relaxing kappa with those rates is therefore the
// same linear map as T^-1 K T (exact up to rounding).  The forcing is folded in:
//   f* = f^e + F'/2 + T^-1 (I - K) T (f - f^e + F'/2)
// which equals f - T^-1 K T (f - f^e) + T^-1 (I - K/2) T F' (Eqs. (11) and (28)).
//
// With the paper's rates s3 = s4 = s5 = s6 = 1 (Section II, below Eq. (17)), (I - K) removes
// every central moment of order three and above, so f* depends on f only through its
// moments of order <= 2: mass, momentum and the raw second moment Pi(f).  Those of f^e and
// F' have closed forms (Pi(f^e) = rho c_s^2 I + rho u u + nu (u g + g u + (u.g) I) with
// c_s^2 = 9(1 - alpha)/19 and g = grad rho; Pi(F') = u F + F u), so collide_kernel needs no
// per-direction Delta and no forward transform; it inverts the ten surviving central
// moments with the same 1-D sweeps.  collide_general_kernel keeps the full 27-moment path
// for any other rates.
#include "lbcm_device.cuh"
#include "lbcm_internal.h"
#include "lbcm_node.cuh"

namespace lbcm {

// ------------------------------------------------------------------ boundary planes
//   z = 0 (inlet or free-slip bottom): the 9 incoming c_z = +1 populations -> zin
//   z = N free-slip top: the 9 incoming c_z = -1 populations -> zout
//   z = N convective: hist(t+1) from hist(t) and the post-stream f(N-1, t+1) (Section IV.A)
// Two kernels with the same results up to the order of the outflow velocity's sums.
// boundary_plane_kernel: one warp per (x, y) column, lane i < 27 handles direction i.  Many
// warps with few instructions each: the faster of the two on planes of fewer than
// kColumnKernelPlane columns.
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int S>
__global__ void __launch_bounds__(128) boundary_plane_kernel(StepArgs a) {
    const int lane = threadIdx.x & 31;
    const long long col = (long long)blockIdx.x * 4 + (threadIdx.x >> 5);
    if (col >= a.plane) return;  // whole warps leave together
    const int x = (int)(col % a.nx), y = (int)(col / a.nx);
    const long long P = a.plane, pxy = col;
    const int N = a.nz - 1;
    const int i = lane < 27 ? lane : 0;
    const int cxi = cx(i), cyi = cy(i), czi = cz(i);
    const bool mine = lane < 27;
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

    if ((a.bc_zlo == BC_INLET || a.bc_zlo == BC_FREESLIP) && mine && czi == 1) {
        float vr, vb;
        if (a.bc_zlo == BC_INLET && a.disc[(long long)ys * a.nx + xs]) {
            // red equilibrium f^e(rho_r0, u_in) with alpha_r and Phi = 0, no blue
            InletVel iv;
            inlet_velocity(a.u_in, a.noise_amp, a.fourier, a.xc, a.yc, a.seed, a.step, xs, ys, a.nx, a.ny, iv);
            const float cu = (float)cxs * iv.ux + (float)cys * iv.uy + (float)czi * iv.uz;
            const float usq = iv.ux * iv.ux + iv.uy * iv.uy + iv.uz * iv.uz;
            vr = a.rho_r0 * (varphi(i, a.alpha_r, a.oma_r) + wgt(i) * eq_poly(cu, usq));
            vb = 0.0f;
        } else {  // half-way specular reflection at z = -1/2
            const float2 v = load_pop<S>(a, mirror_z(ii), ys * a.nx + xs, reader_shift<S>(a, (int)pxy));
            vr = v.x;
            vb = v.y;
        }
        a.zin[(long long)zrank(i) * P + pxy] = vr;
        a.zin[(long long)(9 + zrank(i)) * P + pxy] = vb;
    }
    if (a.bc_zhi == BC_FREESLIP && mine && czi == -1) {
        const float2 v = load_pop<S>(a, mirror_z(ii), (N * a.ny + ys) * a.nx + xs,
                                     reader_shift<S>(a, N * (int)P + (int)pxy));
        a.zout[(long long)zrank(i) * P + pxy] = v.x;
        a.zout[(long long)(9 + zrank(i)) * P + pxy] = v.y;
    }
    if (a.bc_zhi == BC_CONVECTIVE) {
        // post-stream populations of node (x, y, N-1) at t+1 (N-1 >= 1: plain pulls)
        const int z = N - 1;
        float fr = 0.0f, fb = 0.0f;
        if (mine) {
            const int zs = z - czi;
            const float2 v = load_pop<S>(a, ii, (zs * a.ny + ys) * a.nx + xs, reader_shift<S>(a, z * (int)P + (int)pxy));
            fr = v.x;
            fb = v.y;
        }
        const float s_ = fr + fb;
        const float rho = warp_sum_f(s_), jz = warp_sum_f((float)czi * s_);
        const float Fz = (rho - a.rho_b0) * a.gz;
        float lam = (jz + 0.5f * Fz) / rho;  // u_z(x, y, N-1, t+1), Eq. (13)
        lam = fminf(fmaxf(lam, 0.0f), 1.0f);
        const float inv = 1.0f / (1.0f + lam);
        if (mine) {
            const long long hr = (long long)i * P + pxy, hb = (long long)(27 + i) * P + pxy;
            a.hist_out[hr] = (__ldg(a.hist_in + hr) + lam * fr) * inv;
            a.hist_out[hb] = (__ldg(a.hist_in + hb) + lam * fb) * inv;
            if (a.fm_out) {
                a.fm_out[hr] = fr;
                a.fm_out[hb] = fb;
            }
        }
    }
}

// boundary_column_kernel: one thread per (x, y) column, looping over the directions, so that
// the loads and stores of a warp are consecutive columns of one direction's plane; on large
// planes it takes half the time of the warp-per-column kernel (measured on the 256 x 256
// plane: 0.023 against 0.050 ms), on small ones it has too few threads.
constexpr long long kColumnKernelPlane = 24576;
template <int S>
__global__ void __launch_bounds__(128) boundary_column_kernel(StepArgs a) {
    const long long col = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= a.plane) return;
    const int x = (int)(col % a.nx), y = (int)(col / a.nx);
    const long long P = a.plane, pxy = col;
    const int N = a.nz - 1;
    // source column x - c_x, y - c_y of a pull for c = -1, 0, +1, reflected onto the node's own
    // column at a free-slip side wall (where the direction leaving the source has that
    // component reversed: rx / ry)
    int xs3[3], ys3[3];
    bool rx3[3], ry3[3];
#pragma unroll
    for (int d = -1; d <= 1; ++d) {
        int xs = x - d, ys = y - d;
        bool rx = false, ry = false;
        if (xs < 0 || xs >= a.nx) {
            if (a.wall_x) { xs = x; rx = true; } else xs = wrapi(xs, a.nx);
        }
        if (ys < 0 || ys >= a.ny) {
            if (a.wall_y) { ys = y; ry = true; } else ys = wrapi(ys, a.ny);
        }
        xs3[d + 1] = xs; ys3[d + 1] = ys; rx3[d + 1] = rx; ry3[d + 1] = ry;
    }

    if (a.bc_zlo == BC_INLET || a.bc_zlo == BC_FREESLIP) {
        const Own own = reader_shift<S>(a, (int)pxy);
#pragma unroll
        for (int i = 1; i < 27; ++i) {
            if (cz(i) != 1) continue;
            const int xs = xs3[cx(i) + 1], ys = ys3[cy(i) + 1];
            const int cxs = rx3[cx(i) + 1] ? -cx(i) : cx(i), cys = ry3[cy(i) + 1] ? -cy(i) : cy(i);
            float vr, vb;
            if (a.bc_zlo == BC_INLET && a.disc[(long long)ys * a.nx + xs]) {
                // red equilibrium f^e(rho_r0, u_in) with alpha_r and Phi = 0, no blue
                InletVel iv;
                inlet_velocity(a.u_in, a.noise_amp, a.fourier, a.xc, a.yc, a.seed, a.step, xs, ys, a.nx, a.ny, iv);
                const float cu = (float)cxs * iv.ux + (float)cys * iv.uy + iv.uz;
                const float usq = iv.ux * iv.ux + iv.uy * iv.uy + iv.uz * iv.uz;
                vr = a.rho_r0 * (varphi(i, a.alpha_r, a.oma_r) + wgt(i) * eq_poly(cu, usq));
                vb = 0.0f;
            } else {  // half-way specular reflection at z = -1/2
                const float2 v = load_pop<S>(a, mirror_z(i), ys * a.nx + xs, own, mirror_z(dir_of(cxs, cys, 1)));
                vr = v.x;
                vb = v.y;
            }
            a.zin[(long long)zrank(i) * P + pxy] = vr;
            a.zin[(long long)(9 + zrank(i)) * P + pxy] = vb;
        }
    }
    if (a.bc_zhi == BC_FREESLIP) {
        const Own own = reader_shift<S>(a, N * (int)P + (int)pxy);
#pragma unroll
        for (int i = 1; i < 27; ++i) {
            if (cz(i) != -1) continue;
            const int xs = xs3[cx(i) + 1], ys = ys3[cy(i) + 1];
            const int cxs = rx3[cx(i) + 1] ? -cx(i) : cx(i), cys = ry3[cy(i) + 1] ? -cy(i) : cy(i);
            const float2 v = load_pop<S>(a, mirror_z(i), (N * a.ny + ys) * a.nx + xs, own, mirror_z(dir_of(cxs, cys, -1)));
            a.zout[(long long)zrank(i) * P + pxy] = v.x;
            a.zout[(long long)(9 + zrank(i)) * P + pxy] = v.y;
        }
    }
    if (a.bc_zhi == BC_CONVECTIVE) {
        // post-stream populations of node (x, y, N-1) at t+1 (N-1 >= 1: plain pulls)
        const int z = N - 1;
        const Own own = reader_shift<S>(a, z * (int)P + (int)pxy);
        float fr[27], fb[27];
        float rho = 0.0f, jz = 0.0f;
#pragma unroll
        for (int i = 0; i < 27; ++i) {
            const int xs = xs3[cx(i) + 1], ys = ys3[cy(i) + 1];
            const int cxs = rx3[cx(i) + 1] ? -cx(i) : cx(i), cys = ry3[cy(i) + 1] ? -cy(i) : cy(i);
            const float2 v = load_pop<S>(a, i, ((z - cz(i)) * a.ny + ys) * a.nx + xs, own, dir_of(cxs, cys, cz(i)));
            fr[i] = v.x;
            fb[i] = v.y;
        }
#pragma unroll
        for (int i = 0; i < 27; ++i) {
            const float s_ = fr[i] + fb[i];
            rho += s_;
            if (cz(i) > 0) jz += s_; else if (cz(i) < 0) jz -= s_;
        }
        const float Fz = (rho - a.rho_b0) * a.gz;
        float lam = (jz + 0.5f * Fz) / rho;  // u_z(x, y, N-1, t+1), Eq. (13)
        lam = fminf(fmaxf(lam, 0.0f), 1.0f);
        const float inv = 1.0f / (1.0f + lam);
#pragma unroll
        for (int i = 0; i < 27; ++i) {
            const long long hr = (long long)i * P + pxy, hb = (long long)(27 + i) * P + pxy;
            a.hist_out[hr] = (__ldg(a.hist_in + hr) + lam * fr[i]) * inv;
            a.hist_out[hb] = (__ldg(a.hist_in + hb) + lam * fb[i]) * inv;
            if (a.fm_out) {
                a.fm_out[hr] = fr[i];
                a.fm_out[hb] = fb[i];
            }
        }
    }
}

// The boundary planes of a step, with the kernel that suits the plane size.
template <int S>
static void launch_boundary(const StepArgs &a, cudaStream_t s) {
    if (a.plane >= kColumnKernelPlane)
        boundary_column_kernel<S><<<(unsigned)((a.plane + 127) / 128), 128, 0, s>>>(a);
    else
        boundary_plane_kernel<S><<<(unsigned)((a.plane + 3) / 4), 128, 0, s>>>(a);
}

// --------------------------------------------------------------- phase field (K_A)
template <int S, bool W>
__device__ __forceinline__ void phase_field_node(const StepArgs &a) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= a.nx || y >= a.ny) return;
    const Nbr nb(a, x, y, z);
    float fr[27], fb[27];
    gather<S, W>(a, nb, z, fr, fb);
    MassAcc mr, mb;
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        mr.add(i, fr[i]);
        mb.add(i, fb[i]);
    }
    const float rr = mr.total(), rb = mb.total();
    const float ph = order_parameter(rr, rb, a.inv_rho_r0, a.inv_rho_b0);
    if constexpr (S == STORE_FP32) {
        a.phase[nb.n] = make_float2(ph, rr + rb);
    } else if constexpr (S == STORE_FP16) {
        a.ph_cur[nb.n] = make_float4(ph, rr + rb, rr, rb);  // also the FP16 shift densities of S(t+1)
    } else {  // the prediction S(t+1) is encoded against
        a.ph_cur[nb.n] = pack_fit_entry(ph, rr + rb, fit_even(a, rr, rb, ph), fit_odd_fp8(a, fr, fb));
    }
}

// Lattices without side walls (and FP32 with them); and, with separate register bounds, the
// FP16 encodings on lattices with side walls.  Measured on the 240x240x1200 UT lattice: FP16
// 1.97 -> 1.80 ms with a one-block bound, FP16_FIT 3.12 -> 2.52 ms with five; FP32 went the
// other way (2.17 -> 2.69 ms) and keeps the plain bound.
template <int S, bool W>
__global__ void __launch_bounds__(128) phase_field_kernel(StepArgs a) {
    phase_field_node<S, W>(a);
}
template <int S>
__global__ void __launch_bounds__(128, S == STORE_FP16_FIT ? 5 : 1) phase_field_wall_kernel(StepArgs a) {
    phase_field_node<S, true>(a);
}

// ------------------------------------------- moment pass (K_A with the paper's rates)
// With s3 = s4 = s5 = s6 = 1 the collision needs only a node's colour densities, mass,
// momentum and raw second moment (see the header), so the one pull gather of a step happens
// here: the node's phase entry (as phase_field_kernel writes it) plus its 12 collision
// moments go to a.mom, and collide_kernel reads those instead of gathering again.
template <int S, bool W, bool kKeep>
__device__ __forceinline__ void moment_at(const StepArgs &a, int x, int y, int z, unsigned long long pol) {
    const Nbr nb(a, x, y, z);
    float fr[27], fb[27];
    if (z == 0 || z == a.nz - 1)
        gather<S, W, true>(a, nb, z, fr, fb);
    else
        gather<S, W, false>(a, nb, z, fr, fb);
    Moments mo;
    moments_of(fr, fb, mo);
    const float rr = mo.rho_r, rb = mo.rho_b;
    const float ph = order_parameter(rr, rb, a.inv_rho_r0, a.inv_rho_b0);
    if constexpr (S == STORE_FP32) {
        a.phase[nb.n] = make_float2(ph, rr + rb);
    } else if constexpr (S == STORE_FP16) {
        a.ph_cur[nb.n] = make_float4(ph, rr + rb, rr, rb);
    } else {
        a.ph_cur[nb.n] = pack_fit_entry(ph, rr + rb, fit_even(a, rr, rb, ph), fit_odd_fp8(a, fr, fb));
    }
    if constexpr (kKeep)
        store_moments_keep(a.mom, (size_t)a.NN, nb.n, mo, pol);
    else
        store_moments(a.mom, (size_t)a.NN, nb.n, mo);
}

template <int S, bool W>
__device__ __forceinline__ void moment_node(const StepArgs &a) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z + a.z_base;
    if (x >= a.nx || y >= a.ny) return;
    moment_at<S, W, false>(a, x, y, z, 0ull);
}

template <int S, bool W>
__global__ void __launch_bounds__(128) moment_kernel(StepArgs a) {
    moment_node<S, W>(a);
}
template <int S>
__global__ void __launch_bounds__(128, S == STORE_FP16_FIT ? 5 : 1) moment_wall_kernel(StepArgs a) {
    moment_node<S, true>(a);
}

// 1-D shifted moment sweep: values at c = -1, 0, +1 -> central moments of order 0, 1, 2
// about u:  m0 = sum v, m1 = sum v (c - u), m2 = sum v (c - u)^2.
__device__ __forceinline__ void sweep_fwd(float &a0, float &a1, float &a2, float u) {
    const float r0 = a0 + a1 + a2, r1 = a2 - a0, r2 = a2 + a0;
    a0 = r0;
    a1 = fmaf(-u, r0, r1);
    a2 = fmaf(u, fmaf(u, r0, -2.0f * r1), r2);
}
// Inverse of sweep_fwd: raw moments r1 = m1 + u m0, r2 = m2 + 2u m1 + u^2 m0, then
// v0 = r0 - r2, v+ = (r2 + r1)/2, v- = (r2 - r1)/2.
__device__ __forceinline__ void sweep_inv(float &a0, float &a1, float &a2, float u) {
    const float r0 = a0;
    const float r1 = fmaf(u, a0, a1);
    const float r2 = fmaf(u, fmaf(u, a0, 2.0f * a1), a2);
    a1 = r0 - r2;
    a0 = 0.5f * (r2 - r1);
    a2 = 0.5f * (r2 + r1);
}

// ------------------------- collide, perturb, recolour (K_B), any relaxation rates
template <int S, bool W>
__global__ void __launch_bounds__(128) collide_general_kernel(StepArgs a) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= a.nx || y >= a.ny) return;
    const Nbr nb(a, x, y, z);

    // post-stream populations, colour-blind sum and densities (same order as K_A)
    float f[27];
    float rho_r, rho_b;
    {
        float fr[27], fb[27];
        gather<S, W>(a, nb, z, fr, fb);
        MassAcc mr, mb;
#pragma unroll
        for (int i = 0; i < 27; ++i) {
            mr.add(i, fr[i]);
            mb.add(i, fb[i]);
            f[i] = fr[i] + fb[i];
        }
        rho_r = mr.total();
        rho_b = mb.total();
    }

    float gpx, gpy, gpz, grx, gry, grz;
    stencil_gradients<S>(a, nb, z, gpx, gpy, gpz, grx, gry, grz);

    // macroscopic velocity with the Guo half-force (Eq. (13)), body force Eq. (48)
    const float rho = rho_r + rho_b;
    const float inv_rho = 1.0f / rho;
    const float Fx = (rho - a.rho_b0) * a.gx, Fy = (rho - a.rho_b0) * a.gy, Fz = (rho - a.rho_b0) * a.gz;
    float jx = 0.0f, jy = 0.0f, jz = 0.0f;
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        if (cx(i) != 0) jx += (float)cx(i) * f[i];
        if (cy(i) != 0) jy += (float)cy(i) * f[i];
        if (cz(i) != 0) jz += (float)cz(i) * f[i];
    }
    const float ux = (jx + 0.5f * Fx) * inv_rho, uy = (jy + 0.5f * Fy) * inv_rho, uz = (jz + 0.5f * Fz) * inv_rho;

    // order parameter (Eq. (23)) and mixture parameters
    const float phi = order_parameter(rho_r, rho_b, a.inv_rho_r0, a.inv_rho_b0);
    const float hp = 0.5f * (1.0f + phi), hm = 0.5f * (1.0f - phi);
    const float one_m_alpha = one_minus_alpha_bar(a.alpha_mix, rho_r, rho_b, inv_rho, hp, hm, a.oma_r, a.oma_b);
    const float alpha = 1.0f - one_m_alpha;
    const float nu = 1.0f / (hp * a.inv_nu_r + hm * a.inv_nu_b);  // harmonic mean
    const float tau = 3.0f * nu + 0.5f;                           // Eq. (16): 1/s_2nu
    const float s2nu = 1.0f / tau;
    const float Acoef = 2.25f * a.sigma / tau;                     // Eq. (32): A = 9 sigma / (4 tau)

    const float usq = ux * ux + uy * uy + uz * uz;
    const float ugr = ux * grx + uy * gry + uz * grz;
    const float uF = ux * Fx + uy * Fy + uz * Fz;

    // Delta = f - f^e + F'/2, scattered into the tensor-product layout
    float m[27];
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        const float cu = (float)cx(i) * ux + (float)cy(i) * uy + (float)cz(i) * uz;
        const float cg = (float)cx(i) * grx + (float)cy(i) * gry + (float)cz(i) * grz;
        const float cF = (float)cx(i) * Fx + (float)cy(i) * Fy + (float)cz(i) * Fz;
        const float Phi = csq(i) == 0 ? -3.0f * nu * ugr : phi_corr(i) * nu * cu * cg;
        const float fe = rho * fmaf(wgt(i), eq_poly(cu, usq), varphi(i, alpha, one_m_alpha)) + Phi;
        const float Fp = wgt(i) * (3.0f * (cF - uF) + 9.0f * cu * cF);
        m[cell(i)] = f[i] - fe + 0.5f * Fp;
    }

    // forward central-moment transform: z, then y, then x sweeps
#pragma unroll
    for (int p = 0; p < 9; ++p) sweep_fwd(m[p * 3 + 0], m[p * 3 + 1], m[p * 3 + 2], uz);
#pragma unroll
    for (int a0 = 0; a0 < 3; ++a0)
#pragma unroll
        for (int c = 0; c < 3; ++c) sweep_fwd(m[a0 * 9 + 0 + c], m[a0 * 9 + 3 + c], m[a0 * 9 + 6 + c], uy);
#pragma unroll
    for (int q = 0; q < 9; ++q) sweep_fwd(m[q], m[9 + q], m[18 + q], ux);

    // relaxation: kappa <- (I - K') kappa, K' = K in the tensor-product basis
    {
#define KAP(p, q, r) m[(p) * 9 + (q) * 3 + (r)]
        const float o0 = 1.0f - a.s0, o1 = 1.0f - a.s1, o2 = 1.0f - s2nu, o2b = 1.0f - a.s2b;
        const float o3 = 1.0f - a.s3, o4 = 1.0f - a.s4, o5 = 1.0f - a.s5, o6 = 1.0f - a.s6;
        KAP(0, 0, 0) *= o0;
        KAP(1, 0, 0) *= o1; KAP(0, 1, 0) *= o1; KAP(0, 0, 1) *= o1;
        KAP(1, 1, 0) *= o2; KAP(1, 0, 1) *= o2; KAP(0, 1, 1) *= o2;
        {
            const float tr = KAP(2, 0, 0) + KAP(0, 2, 0) + KAP(0, 0, 2);
            const float d1 = KAP(2, 0, 0) - KAP(0, 2, 0), d2 = KAP(2, 0, 0) - KAP(0, 0, 2);
            const float t = o2b * tr, e1 = o2 * d1, e2 = o2 * d2;
            const float third = 1.0f / 3.0f;
            KAP(2, 0, 0) = (t + e1 + e2) * third;
            KAP(0, 2, 0) = (t - 2.0f * e1 + e2) * third;
            KAP(0, 0, 2) = (t + e1 - 2.0f * e2) * third;
        }
        KAP(2, 1, 0) *= o3; KAP(2, 0, 1) *= o3; KAP(1, 2, 0) *= o3; KAP(0, 2, 1) *= o3;
        KAP(1, 0, 2) *= o3; KAP(0, 1, 2) *= o3; KAP(1, 1, 1) *= o3;
        KAP(2, 2, 0) *= o4; KAP(2, 0, 2) *= o4; KAP(0, 2, 2) *= o4;
        KAP(2, 1, 1) *= o4; KAP(1, 2, 1) *= o4; KAP(1, 1, 2) *= o4;
        KAP(2, 2, 1) *= o5; KAP(2, 1, 2) *= o5; KAP(1, 2, 2) *= o5;
        KAP(2, 2, 2) *= o6;
#undef KAP
    }

    // inverse transform: x, then y, then z sweeps
#pragma unroll
    for (int q = 0; q < 9; ++q) sweep_inv(m[q], m[9 + q], m[18 + q], ux);
#pragma unroll
    for (int a0 = 0; a0 < 3; ++a0)
#pragma unroll
        for (int c = 0; c < 3; ++c) sweep_inv(m[a0 * 9 + 0 + c], m[a0 * 9 + 3 + c], m[a0 * 9 + 6 + c], uy);
#pragma unroll
    for (int p = 0; p < 9; ++p) sweep_inv(m[p * 3 + 0], m[p * 3 + 1], m[p * 3 + 2], uz);

    // perturbation (Eq. (30), squared numerator, both colours) and recolouring
    const float g2 = gpx * gpx + gpy * gpy + gpz * gpz;
    const float inv_gm = 1.0f / sqrtf(g2 + a.eps2);  // 1/|grad phi|_eps
    const float frac_r = rho_r * inv_rho, frac_b = rho_b * inv_rho;
    const float seg0 = a.beta * rho_r * rho_b * inv_rho * inv_gm;  // beta rho_r rho_b / (rho |g|)
    const float pert = Acoef * inv_gm;
    const int n = nb.n;
    MassAcc sum_r, sum_b;  // moving populations written (as read back), per colour
#pragma unroll
    for (int i = 1; i < 27; ++i) {  // the rest direction is the per-colour remainder below
        const float cu = (float)cx(i) * ux + (float)cy(i) * uy + (float)cz(i) * uz;
        const float cg = (float)cx(i) * grx + (float)cy(i) * gry + (float)cz(i) * grz;
        const float cF = (float)cx(i) * Fx + (float)cy(i) * Fy + (float)cz(i) * Fz;
        const float Phi = phi_corr(i) * nu * cu * cg;
        const float fe = rho * fmaf(wgt(i), eq_poly(cu, usq), varphi(i, alpha, one_m_alpha)) + Phi;
        const float Fp = wgt(i) * (3.0f * (cF - uF) + 9.0f * cu * cF);
        const float cgp = (float)cx(i) * gpx + (float)cy(i) * gpy + (float)cz(i) * gpz;
        float fs = fe + 0.5f * Fp + m[cell(i)];
        fs += pert * (wgt(i) * cgp * cgp - bcoef(i) * g2);
        const float seg = seg0 * varphi(i, alpha, one_m_alpha) * cgp * inv_cnorm(i);
        const float2 d = store_pop<S>(a, i, n, make_float2(fmaf(frac_r, fs, seg), fmaf(frac_b, fs, -seg)),
                                      dest_shift<S>(a, nb, i));
        sum_r.add(i, d.x);
        sum_b.add(i, d.y);
    }
    // rest direction as the per-colour remainder (see collide_from_moments)
    store_pop<S>(a, 0, n, make_float2(rho_r - sum_r.s, rho_b - sum_b.s), no_shift());
}


// Collision, perturbation and recolouring of one node from its moments and gradients;
// writes the 54 post-collision populations of node n.
template <bool kForce, int S>
__device__ __forceinline__ void collide_from_moments(const StepArgs &a, const Nbr &nb, const Moments &mo, float gpx,
                                                     float gpy, float gpz, float grx, float gry, float grz) {
    const int n = nb.n;
    const float rho_r = mo.rho_r, rho_b = mo.rho_b, sf = mo.sf, jx = mo.jx, jy = mo.jy, jz = mo.jz;
    const float pxx = mo.pxx, pyy = mo.pyy, pzz = mo.pzz, pxy = mo.pxy, pxz = mo.pxz, pyz = mo.pyz;
    // macroscopic quantities (Eqs. (13), (48), (23)) and mixture parameters
    const float rho = rho_r + rho_b;
    const float inv_rho = 1.0f / rho;
    float Fx = 0.0f, Fy = 0.0f, Fz = 0.0f;
    if (kForce) {
        const float fo = rho - a.rho_b0;
        Fx = fo * a.gx; Fy = fo * a.gy; Fz = fo * a.gz;
    }
    const float jFx = fmaf(0.5f, Fx, jx), jFy = fmaf(0.5f, Fy, jy), jFz = fmaf(0.5f, Fz, jz);
    const float ux = jFx * inv_rho, uy = jFy * inv_rho, uz = jFz * inv_rho;
    const float phi = order_parameter(rho_r, rho_b, a.inv_rho_r0, a.inv_rho_b0);
    const float hp = 0.5f * (1.0f + phi), hm = 0.5f * (1.0f - phi);
    const float oma = one_minus_alpha_bar(a.alpha_mix, rho_r, rho_b, inv_rho, hp, hm, a.oma_r, a.oma_b);
    const float alpha = 1.0f - oma;
    const float nu = 1.0f / (hp * a.inv_nu_r + hm * a.inv_nu_b);
    const float tau = 3.0f * nu + 0.5f;
    const float s2nu = 1.0f / tau;
    const float Acoef = 2.25f * a.sigma / tau;  // A = 9 sigma / (4 tau)
    const float usq = ux * ux + uy * uy + uz * uz;
    const float ugr = ux * grx + uy * gry + uz * grz;
    const float uF = ux * Fx + uy * Fy + uz * Fz;

    // moments of Delta = f - f^e + F'/2: mass, momentum, raw second moment
    const float M = sf - rho;
    const float dx = fmaf(-rho, ux, jFx), dy = fmaf(-rho, uy, jFy), dz = fmaf(-rho, uz, jFz);
    const float cs2r = rho * oma * (9.0f / 19.0f);
    float Dxx = pxx - (cs2r + rho * ux * ux + nu * (2.0f * ux * grx + ugr));
    float Dyy = pyy - (cs2r + rho * uy * uy + nu * (2.0f * uy * gry + ugr));
    float Dzz = pzz - (cs2r + rho * uz * uz + nu * (2.0f * uz * grz + ugr));
    float Dxy = pxy - (rho * ux * uy + nu * (ux * gry + uy * grx));
    float Dxz = pxz - (rho * ux * uz + nu * (ux * grz + uz * grx));
    float Dyz = pyz - (rho * uy * uz + nu * (uy * grz + uz * gry));
    if (kForce) {
        Dxx += ux * Fx; Dyy += uy * Fy; Dzz += uz * Fz;
        Dxy += 0.5f * (ux * Fy + uy * Fx); Dxz += 0.5f * (ux * Fz + uz * Fx); Dyz += 0.5f * (uy * Fz + uz * Fy);
    }
    // central moments of Delta, then (I - K') applied
    const float k000 = (1.0f - a.s0) * M;
    const float o1 = 1.0f - a.s1;
    const float k100 = o1 * fmaf(-ux, M, dx), k010 = o1 * fmaf(-uy, M, dy), k001 = o1 * fmaf(-uz, M, dz);
    const float o2 = 1.0f - s2nu;
    const float cxx = Dxx - 2.0f * ux * dx + ux * ux * M;
    const float cyy = Dyy - 2.0f * uy * dy + uy * uy * M;
    const float czz = Dzz - 2.0f * uz * dz + uz * uz * M;
    const float k110 = o2 * (Dxy - ux * dy - uy * dx + ux * uy * M);
    const float k101 = o2 * (Dxz - ux * dz - uz * dx + ux * uz * M);
    const float k011 = o2 * (Dyz - uy * dz - uz * dy + uy * uz * M);
    float k200, k020, k002;
    {
        const float t = (1.0f - a.s2b) * (cxx + cyy + czz);
        const float e1 = o2 * (cxx - cyy), e2 = o2 * (cxx - czz);
        const float third = 1.0f / 3.0f;
        k200 = (t + e1 + e2) * third;
        k020 = (t - 2.0f * e1 + e2) * third;
        k002 = (t + e1 - 2.0f * e2) * third;
    }

    // inverse transform of the ten surviving moments: z sweep, y sweep (x sweep per direction)
    const InvAxis Ax(ux), Ay(uy), Az(uz);
    // z sweep of the columns (p, q): values V_pq[cz]
    float V00[3], V10[3], V01[3], V20[3], V02[3], V11[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        V00[c] = fmaf(Az.g0[c], k000, fmaf(Az.g1[c], k001, g2c(c - 1) * k002));
        V10[c] = fmaf(Az.g0[c], k100, Az.g1[c] * k101);
        V01[c] = fmaf(Az.g0[c], k010, Az.g1[c] * k011);
        V20[c] = Az.g0[c] * k200;
        V02[c] = Az.g0[c] * k020;
        V11[c] = Az.g0[c] * k110;
    }
    // y sweep: W_p[cy][cz]
    float W0[3][3], W1[3][3], W2[3][3];
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            W0[b][c] = fmaf(Ay.g0[b], V00[c], fmaf(Ay.g1[b], V01[c], g2c(b - 1) * V02[c]));
            W1[b][c] = fmaf(Ay.g0[b], V10[c], Ay.g1[b] * V11[c]);
            W2[b][c] = Ay.g0[b] * V20[c];
        }

    // perturbation (Eq. (30), squared numerator, both colours) and recolouring
    const float g2 = gpx * gpx + gpy * gpy + gpz * gpz;
    const float inv_gm = 1.0f / sqrtf(g2 + a.eps2);  // 1/|grad phi|_eps
    const float pert = Acoef * inv_gm;
    const float frac_r = rho_r * inv_rho, frac_b = rho_b * inv_rho;
    const float seg0 = a.beta * rho_r * rho_b * inv_rho * inv_gm;
    // moving populations written (as read back), per colour, summed as MassAcc sums them
    float2 sum = make_float2(0.0f, 0.0f);
    const float2 frac = make_float2(frac_r, frac_b);
    // opposite pairs (i, i+1), c_{i+1} = -c_i: c.u, c.grad rho and c.grad phi change sign;
    // f^e splits into an even part (rest weight, quadratic terms, Phi) and an odd part
    // (linear and cubic terms), the perturbation is even and the recolouring flux odd.
#pragma unroll
    for (int i = 1; i < 27; i += 2) {
        const float cu = (float)cx(i) * ux + (float)cy(i) * uy + (float)cz(i) * uz;
        const float cgr = (float)cx(i) * grx + (float)cy(i) * gry + (float)cz(i) * grz;
        const float cgp = (float)cx(i) * gpx + (float)cy(i) * gpy + (float)cz(i) * gpz;
        const float h = 4.5f * cu;
        const float ev = fmaf(h, cu, -1.5f * usq);                  // 9/2 cu^2 - 3/2 u^2
        const float od = cu * fmaf(h, cu, fmaf(-4.5f, usq, 3.0f));  // 3 cu + 9/2 cu^3 - 9/2 cu u^2
        const float rw = rho * wgt(i);
        float even = fmaf(rw, ev, rho * varphi(i, alpha, oma));
        even = fmaf(phi_corr(i) * nu * cu, cgr, even);                // Phi_i
        even = fmaf(pert, wgt(i) * cgp * cgp - bcoef(i) * g2, even);  // perturbation
        float odd = rw * od;
        if (kForce) {
            const float cF = (float)cx(i) * Fx + (float)cy(i) * Fy + (float)cz(i) * Fz;
            even = fmaf(0.5f * wgt(i), fmaf(9.0f * cu, cF, -3.0f * uF), even);  // F'/2, even part
            odd = fmaf(1.5f * wgt(i), cF, odd);                                   // F'/2, odd part
        }
        const int X = cx(i) + 1, Y = cy(i) + 1, Z = cz(i) + 1;
        const float rp = fmaf(Ax.g0[X], W0[Y][Z], fmaf(Ax.g1[X], W1[Y][Z], g2c(cx(i)) * W2[Y][Z]));
        const float rm = fmaf(Ax.g0[2 - X], W0[2 - Y][2 - Z], fmaf(Ax.g1[2 - X], W1[2 - Y][2 - Z], g2c(cx(i)) * W2[2 - Y][2 - Z]));
        const float fsp = (even + odd) + rp, fsm = (even - odd) + rm;
        const float seg = seg0 * varphi(i, alpha, oma) * inv_cnorm(i) * cgp;
        if constexpr (S == STORE_FP32) {
            // both colours at once: packed FP32x2 operations, each lane rounded as the scalar
            // ones (measured 2% faster for FP32, slower for the half-precision encodings)
            const float2 vp = __ffma2_rn(frac, make_float2(fsp, fsp), make_float2(seg, -seg));
            const float2 vm = __ffma2_rn(frac, make_float2(fsm, fsm), make_float2(-seg, seg));
            store_pop<S>(a, i, n, vp, no_shift());
            store_pop<S>(a, i + 1, n, vm, no_shift());
            sum = __fadd2_rn(sum, __fadd2_rn(vp, vm));
        } else {
            const float2 dp_ = store_pop<S>(a, i, n, make_float2(fmaf(frac_r, fsp, seg), fmaf(frac_b, fsp, -seg)),
                                            dest_shift<S>(a, nb, i));
            const float2 dm_ = store_pop<S>(a, i + 1, n, make_float2(fmaf(frac_r, fsm, -seg), fmaf(frac_b, fsm, seg)),
                                            dest_shift<S>(a, nb, i + 1));
            sum.x += dp_.x + dm_.x;
            sum.y += dp_.y + dm_.y;
        }
    }
    const float sum_r = sum.x, sum_b = sum.y;
    // Rest direction.  In exact arithmetic the step keeps each colour's mass at this node
    // (sum_i f_i^k* = rho_k), so the rest population is that mass minus the moving ones as
    // they will be read back; this equals Eqs. (33), (34) for i = 0 and keeps the FP32
    // rounding of the lattice constants and any storage rounding from drifting the colour
    // masses step after step (the pairwise sum above is MassAcc's association).
    store_pop<S>(a, 0, n, make_float2(rho_r - sum_r, rho_b - sum_b), no_shift());
}

// -------- collide, perturb, recolour (K_B) with the paper's rates s3 = s4 = s5 = s6 = 1
// Reads the node's moments from the moment pass (no population gather), takes the
// gradients from the 26 neighbours' phase entries and writes the 54 populations.
// kRec (FP32, adjoint recompute): also writes the node's gradients to a.grad4 / a.grad2 (its
// moments are already in a.mom).
// Blocks per SM (register bound): FP32 6, FP16 5, FP16_FIT 4 (its encoding needs the most
// registers).
template <bool kForce, int S, bool kRec, bool kOnce>
__device__ __forceinline__ void collide_at(const StepArgs &a, int x, int y, int z) {
    const Nbr nb(a, x, y, z);
    const Moments mo = kOnce ? load_moments_once(a.mom, (size_t)a.NN, nb.n) : load_moments(a.mom, (size_t)a.NN, nb.n);
    float gpx, gpy, gpz, grx, gry, grz;
    if (z == 0)
        stencil_gradients<S, true>(a, nb, z, gpx, gpy, gpz, grx, gry, grz);
    else
        stencil_gradients<S, false>(a, nb, z, gpx, gpy, gpz, grx, gry, grz);
    if constexpr (kRec) {
        a.grad4[nb.n] = make_float4(gpx, gpy, gpz, grx);
        a.grad2[nb.n] = make_float2(gry, grz);
    }
    collide_from_moments<kForce, S>(a, nb, mo, gpx, gpy, gpz, grx, gry, grz);
}

template <bool kForce, int S, bool kRec>
__global__ void __launch_bounds__(128, (S == STORE_FP32 ? 6 : (S == STORE_FP16 ? 5 : 4))) collide_kernel(StepArgs a) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z + a.z_base;
    if (x >= a.nx || y >= a.ny) return;
    collide_at<kForce, S, kRec, false>(a, x, y, z);
}

// ------------------------------------------------------- fused step (one launch)
// Both passes of a step in one cooperative launch (params.step_kernel = 1).  The work is a fixed
// sequence of items, each a 32 x kFusedRows tile of one plane: the gathers of a plane are issued
// lag planes before the collisions that read them (FusedCtl::ops), and block b takes items b,
// b + G, b + 2G, ... (G blocks, all resident).  A gather item counts itself into done[z] once its
// writes are visible device-wide; a collision item of plane z waits until planes z - 1, z, z + 1
// are counted complete.  Every item waits only for items earlier in the sequence, held by
// resident blocks that do not wait on it, so the waits end; each is also bounded, and on running
// out it sets f.err (reported by the next synchronising call) and goes on.  With the lag (about
// one round of G items) a collision item seldom waits, and a plane's 48-byte moments are read a
// few planes after they were written: they stay in L2 (stored with the evict-last policy) and,
// read once, their lines are dropped without being written back.  The step then moves close to
// the method's 448 bytes a node from DRAM (450-500 measured, against 522 for the two launches),
// but its blocks wait and synchronise at every item and it streams at a lower fraction of the
// bandwidth: on GB300 it is 3% slower than the two launches on the 256x256x1024 jet and about
// level with them on smaller ones, and the two launches stay the default.
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits until the gathers of planes p0, p1, p2 are all counted complete (the three counters
// are read together).  Bounded by time, kFusedWaitNs, and as a backstop by the number of
// polls; on giving up it sets f.err and returns.
__device__ __forceinline__ void wait_planes(const FusedCtl &f, int p0, int p1, int p2) {
    const unsigned long long t0 = global_ns();
    for (long long k = 0;; ++k) {
        const unsigned long long d0 = ld_acquire_u64(f.done + p0), d1 = ld_acquire_u64(f.done + p1),
                                 d2 = ld_acquire_u64(f.done + p2);
        if (d0 >= f.target && d1 >= f.target && d2 >= f.target) return;
        if (global_ns() - t0 > kFusedWaitNs || k > kFusedSpinLimit) {
            atomicExch(f.err, 1);
            return;
        }
        __nanosleep(64);
    }
}

// The fused kernel's wait on a plane that no gather completes (f.target beyond reach): one
// thread gives up after the wait's limit, sets f.err and records the time it waited in *ns.
__global__ void fused_wait_probe_kernel(FusedCtl f, unsigned long long *ns) {
    if (threadIdx.x != 0) return;
    const unsigned long long t0 = global_ns();
    wait_planes(f, 0, 0, 0);
    *ns = global_ns() - t0;
}

cudaError_t launch_fused_wait_probe(const FusedCtl &f, unsigned long long *ns, cudaStream_t s) {
    fused_wait_probe_kernel<<<1, 32, 0, s>>>(f, ns);
    return cudaGetLastError();
}

template <bool kForce, int S, bool W>
__global__ void __launch_bounds__(128, (S == STORE_FP32 ? 6 : (S == STORE_FP16 ? 5 : 4))) step_kernel(StepArgs a, FusedCtl f) {
    // items are 32 x kFusedRows tiles of a plane, taken by the blocks round-robin; each warp
    // walks kFusedRows / 4 rows of the tile
    const bool lead = threadIdx.x == 0 && threadIdx.y == 0;
    const int T = f.items_x * f.items_y;
    const long long total = (long long)f.nops * T;
    const unsigned long long pol = l2_evict_last_policy();
    for (long long it = blockIdx.x; it < total; it += gridDim.x) {
        const int op = (int)(it / T), t = (int)(it - (long long)op * T);
        const int2 o = f.ops[op];
        const int z = o.y;
        const int x = (t % f.items_x) * 32 + threadIdx.x;
        const int y0 = (t / f.items_x) * kFusedRows;
        if (o.x == 0) {  // gather: phase entries and moments of the tile
#pragma unroll 1
            for (int r = threadIdx.y; r < kFusedRows; r += 4) {
                const int y = y0 + r;
                if (x < a.nx && y < a.ny) moment_at<S, W, true>(a, x, y, z, pol);
            }
            __syncthreads();
            if (lead) {
                __threadfence();
                atomicAdd(f.done + z, 1ull);
            }
        } else {  // collision of the tile, once the three planes of its stencil are gathered
            if (lead) {
                const bool pz = a.bc_zlo == BC_PERIODIC;
                wait_planes(f, z, (z > 0 || pz) ? (z > 0 ? z - 1 : a.nz - 1) : z,
                            (z < a.nz - 1 || pz) ? (z < a.nz - 1 ? z + 1 : 0) : z);
            }
            __syncthreads();
#pragma unroll 1
            for (int r = threadIdx.y; r < kFusedRows; r += 4) {
                const int y = y0 + r;
                const bool in = x < a.nx && y < a.ny;
                if (in) collide_at<kForce, S, false, true>(a, x, y, z);
                if (f.discard) {  // every lane has read its moments: drop the lines
                    __syncwarp();
                    if (in && (threadIdx.x & 7) == 0) {
                        const size_t n = ((size_t)z * a.ny + y) * a.nx + x, NN = (size_t)a.NN;
                        l2_discard(a.mom + n);
                        l2_discard(a.mom + NN + n);
                        l2_discard(a.mom + 2 * NN + n);
                    }
                }
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------ launchers
template <int S, bool W>
static void launch_step_sw(const StepArgs &a, cudaStream_t s, cudaEvent_t *ev, long long *launches, int passes) {
    const bool paper_rates = a.s3 == 1.0f && a.s4 == 1.0f && a.s5 == 1.0f && a.s6 == 1.0f;
    const bool force = a.gx != 0.0f || a.gy != 0.0f || a.gz != 0.0f;
    dim3 blk(32, 4, 1), grd((a.nx + 31) / 32, (a.ny + 3) / 4, a.nz);
    if (passes & PASS_GATHER) {
        if (ev) cudaEventRecord(ev[0], s);
        if (a.bc_zlo != BC_PERIODIC || a.bc_zhi != BC_PERIODIC) {
            launch_boundary<S>(a, s);
            *launches += 1;
        }
        if (ev) cudaEventRecord(ev[1], s);
        // pass 1: the step's pull gather (phase field, and the collision moments when the
        // paper's rates let the collision work from them)
        if (paper_rates) {
            if constexpr (W && S != STORE_FP32)
                moment_wall_kernel<S><<<grd, blk, 0, s>>>(a);
            else
                moment_kernel<S, W><<<grd, blk, 0, s>>>(a);
        } else {
            if constexpr (W && S != STORE_FP32)
                phase_field_wall_kernel<S><<<grd, blk, 0, s>>>(a);
            else
                phase_field_kernel<S, W><<<grd, blk, 0, s>>>(a);
        }
        if (ev) cudaEventRecord(ev[2], s);
        *launches += 1;
    }
    if (!(passes & PASS_COLLIDE)) return;
    // pass 2: the collision, writing S(t+1)
    if (ev && !(passes & PASS_GATHER)) cudaEventRecord(ev[2], s);
    const bool rec = S == STORE_FP32 && a.grad4 != nullptr;  // paper rates only (adjoint)
    if (!paper_rates)
        collide_general_kernel<S, W><<<grd, blk, 0, s>>>(a);
    else if (rec && force)
        collide_kernel<true, S, S == STORE_FP32><<<grd, blk, 0, s>>>(a);
    else if (rec)
        collide_kernel<false, S, S == STORE_FP32><<<grd, blk, 0, s>>>(a);
    else if (force)
        collide_kernel<true, S, false><<<grd, blk, 0, s>>>(a);
    else
        collide_kernel<false, S, false><<<grd, blk, 0, s>>>(a);
    if (ev) cudaEventRecord(ev[3], s);
    *launches += 1;
}

template <bool kForce, int S, bool W>
static cudaError_t launch_fused_sw(const StepArgs &a, const FusedCtl &f, int grid, cudaStream_t s) {
    void *args[] = {(void *)&a, (void *)&f};
    return cudaLaunchCooperativeKernel((const void *)step_kernel<kForce, S, W>, dim3(grid), dim3(32, 4, 1), args, 0, s);
}

template <int S>
static cudaError_t fused_sw(const StepArgs &a, const FusedCtl &f, int grid, cudaStream_t s, int *occ) {
    const bool force = a.gx != 0.0f || a.gy != 0.0f || a.gz != 0.0f;
    const bool walls = a.wall_x || a.wall_y;
    const void *fn = force ? (walls ? (const void *)step_kernel<true, S, true> : (const void *)step_kernel<true, S, false>)
                           : (walls ? (const void *)step_kernel<false, S, true> : (const void *)step_kernel<false, S, false>);
    if (occ) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, fn, 128, 0);
    if (force)
        return walls ? launch_fused_sw<true, S, true>(a, f, grid, s) : launch_fused_sw<true, S, false>(a, f, grid, s);
    return walls ? launch_fused_sw<false, S, true>(a, f, grid, s) : launch_fused_sw<false, S, false>(a, f, grid, s);
}

cudaError_t fused_occupancy(const StepArgs &a, int storage, int *blocks_per_sm) {
    if (storage == STORE_FP16) return fused_sw<STORE_FP16>(a, FusedCtl{}, 0, nullptr, blocks_per_sm);
    if (storage == STORE_FP16_FIT) return fused_sw<STORE_FP16_FIT>(a, FusedCtl{}, 0, nullptr, blocks_per_sm);
    return fused_sw<STORE_FP32>(a, FusedCtl{}, 0, nullptr, blocks_per_sm);
}

cudaError_t launch_fused_step(const StepArgs &a, int storage, const FusedCtl &f, int grid, cudaStream_t s,
                              cudaEvent_t *ev, long long *launches) {
    if (ev) cudaEventRecord(ev[0], s);
    if (a.bc_zlo != BC_PERIODIC || a.bc_zhi != BC_PERIODIC) {
        if (storage == STORE_FP16)
            launch_boundary<STORE_FP16>(a, s);
        else if (storage == STORE_FP16_FIT)
            launch_boundary<STORE_FP16_FIT>(a, s);
        else
            launch_boundary<STORE_FP32>(a, s);
        *launches += 1;
    }
    if (ev) cudaEventRecord(ev[1], s);
    cudaError_t e;
    if (storage == STORE_FP16)
        e = fused_sw<STORE_FP16>(a, f, grid, s, nullptr);
    else if (storage == STORE_FP16_FIT)
        e = fused_sw<STORE_FP16_FIT>(a, f, grid, s, nullptr);
    else
        e = fused_sw<STORE_FP32>(a, f, grid, s, nullptr);
    if (e != cudaSuccess) return e;
    *launches += 1;
    if (ev) {
        cudaEventRecord(ev[2], s);
        cudaEventRecord(ev[3], s);
    }
    return cudaGetLastError();
}

template <int S>
static void launch_step_s(const StepArgs &a, cudaStream_t s, cudaEvent_t *ev, long long *launches, int passes) {
    if (a.wall_x || a.wall_y)
        launch_step_sw<S, true>(a, s, ev, launches, passes);
    else
        launch_step_sw<S, false>(a, s, ev, launches, passes);
}

cudaError_t launch_step(const StepArgs &a, int storage, cudaStream_t s, cudaEvent_t *ev, long long *launches,
                        int passes) {
    if (storage == STORE_FP16)
        launch_step_s<STORE_FP16>(a, s, ev, launches, passes);
    else if (storage == STORE_FP16_FIT)
        launch_step_s<STORE_FP16_FIT>(a, s, ev, launches, passes);
    else
        launch_step_s<STORE_FP32>(a, s, ev, launches, passes);
    return cudaGetLastError();
}

}  // namespace lbcm
