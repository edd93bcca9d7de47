// lbcm_internal.h -- declarations shared by the translation units of the library.
#pragma once
#include <cuda_runtime.h>
#include "lbcm_device.cuh"

namespace lbcm {
// One time step (boundary planes, gather pass, collision) on stream s, for population storage
// STORE_FP32, STORE_FP16 or STORE_FP16_FIT.  passes selects PASS_GATHER (boundary planes and the
// gather pass: phase field and collision moments), PASS_COLLIDE (the collision, which writes
// S(t+1)) or both; a z-slab decomposition exchanges the phase halo between the two.  When ev
// is not NULL, ev[0..3] are recorded before the boundary kernel, before the gather kernel,
// before the collision kernel and after it (those of the passes launched).  *launches is
// increased by the number of kernels launched.
enum { PASS_GATHER = 1, PASS_COLLIDE = 2, PASS_BOTH = 3 };
cudaError_t launch_step(const StepArgs &a, int storage, cudaStream_t s, cudaEvent_t *ev, long long *launches,
                        int passes = PASS_BOTH);

// Control block of the fused step kernel (both passes of a step in one cooperative launch,
// paper rates only): the item sequence and the per-plane completion counters.
struct FusedCtl {
    unsigned long long *done;   // done[z]: gather items of plane z finished, summed over launches
    const int2 *ops;            // (0 gather / 1 collision, plane) in issue order, nops entries
    int *err;                   // set when a wait for a plane's gathers ran out
    unsigned long long target;  // done[z] after this launch has gathered plane z
    int nops, items_x, items_y; // items per row of tiles and rows of tiles of a plane
    int discard;                // the moments' L2 lines may be dropped once read (nx % 32 == 0)
};
constexpr unsigned long long kFusedWaitNs = 1000000000ull;  // a plane wait gives up after 1 s
constexpr long long kFusedSpinLimit = 1ll << 26;            // and after this many polls (> 4 s)
// An item is a 32 x kFusedRows tile of a plane (a multiple of 4: each of the 4 warps walks
// every fourth row); settable at build time.  The lead of the gathers over the collisions is
// host code (lbcm_api.cu).
#ifndef LBCM_FUSED_ROWS
#define LBCM_FUSED_ROWS 32
#endif
constexpr int kFusedRows = LBCM_FUSED_ROWS;
static_assert(kFusedRows % 4 == 0 && kFusedRows >= 4, "fused item rows must be a positive multiple of 4");
// Blocks per SM the fused kernel can keep resident (its cooperative grid is this times the SMs).
cudaError_t fused_occupancy(const StepArgs &a, int storage, int *blocks_per_sm);
// Boundary planes, then the fused kernel on `grid` blocks; ev as for launch_step (the fused
// kernel's time lands between ev[1] and ev[2], the collision's slot stays empty).
cudaError_t launch_fused_step(const StepArgs &a, int storage, const FusedCtl &f, int grid, cudaStream_t s,
                              cudaEvent_t *ev, long long *launches);
// One thread runs the fused kernel's plane wait with f.target out of reach: it gives up after
// the wait's limit and sets *f.err; *ns receives the time it waited.
cudaError_t launch_fused_wait_probe(const FusedCtl &f, unsigned long long *ns, cudaStream_t s);

// Adjoint state and scratch of one reverse step (FP32 populations, paper rates).
//   lp_in / lr_in   lambda of S(n+1): pushed part [27][NN] float2 and deferred density part [NN]
//   lp_out / lr_out the same for S(n)
//   lga, lgb        lambda of (grad phi, grad rho) per node: (gpx, gpy, gpz, grx), (gry, grz)
//   lc              direct lambda of f(N) on a convective top [54][nx ny]
//   li              direct lambda of the red inlet populations that come from the disc [9][nx ny]
//   lh_in / lh_out  lambda of the outflow history hist(n+1) / hist(n) [54][nx ny]
//   acc_coll        FP64 per-block sums of dJ/d(sigma, nu_r, nu_b) [blocks][3]
//   acc_inlet       FP64 per-block sums of dJ/d(u_in, a_1, b_1, ..., a_8, b_8) [blocks][17]
//   mom             the forward step's collision moments per node, [3][NN] float4 as the moment
//                   pass writes them: (rho_r, rho_b, sf, jx), (jy, jz, pxx, pyy), (pzz, pxy, pxz, pyz)
//   grad4, grad2    its gradients per node (as StepArgs::grad4, grad2)
//   fm              the forward step's f(N-1) of the outflow columns [54][nx ny]
struct AdjArgs {
    const float4 *mom, *grad4;
    const float2 *grad2;
    const float *fm;
    const float2 *lp_in, *lr_in;
    float2 *lp_out, *lr_out;
    float4 *lga;
    float2 *lgb;
    float *lc, *li;
    const float *lh_in;
    float *lh_out;
    double *acc_coll, *acc_inlet;
};

// Blocks of the collide-adjoint and boundary-adjoint grids (sizes of acc_coll, acc_inlet).
long long adj_collide_blocks(const StepArgs &a);
long long adj_boundary_blocks(const StepArgs &a);
// Reverse of the step described by a (hist_in / hist_out as the forward step n wrote them;
// its populations are not read: g.mom, g.grad4, g.grad2 and g.fm hold what the reverse needs of
// step n).
cudaError_t launch_adjoint_step(const StepArgs &a, const AdjArgs &g, cudaStream_t s, long long *launches);
// Objective of the state a.pin (0 interface area, args[0] = eps; 1 penetration length,
// args[0] = delta): scalar[0] = J; writes lambda_S(T) into g.lp_out / g.lr_out.
cudaError_t launch_objective(const StepArgs &a, const AdjArgs &g, int objective, const double *args, float2 *ph,
                             float2 *lr_obj, double *acc_obj, double *scalar, cudaStream_t s, long long *launches);
// out[1] = dJ/du_in, out[2..4] = dJ/d(sigma, nu_r, nu_b), out[5..20] = dJ/d(a_1, b_1, ..., b_8).
cudaError_t launch_adjoint_reduce(const AdjArgs &g, long long nblk_coll, long long nblk_inlet, double *out,
                                  cudaStream_t s, long long *launches);
// dJ/dS in the canonical layout [k][i][z][y][x] from (g.lp_in, g.lr_in).
cudaError_t launch_adjoint_state(const StepArgs &a, const AdjArgs &g, float *out, cudaStream_t s, long long *launches);

// Fragment labelling of the state a.pin (stored as `storage`): union-find labels (smallest node
// index of each component, -1 outside the jet), volumes and z = 0 flags at the roots, root
// counts per block of 1024 nodes and their exclusive scan boff[0..nblk] (boff[nblk] = roots).
// count and touch must be zero on entry; err is set if a bounded loop ran out.
cudaError_t launch_fragments_label(const StepArgs &a, int storage, int connectivity, int *label, int *count,
                                   uint8_t *touch, int *bc, long long *boff, int *err, cudaStream_t s,
                                   long long *launches);
// The roots in index order with their volumes and z = 0 flags.
cudaError_t launch_fragments_write(const StepArgs &a, int connectivity, const int *label, const int *count,
                                   const uint8_t *touch, const long long *boff, long long *out_root,
                                   long long *out_vol, uint8_t *out_touch, cudaStream_t s, long long *launches);
}  // namespace lbcm
