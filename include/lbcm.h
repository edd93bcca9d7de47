/*
 * lbcm.h -- C ABI of the GB300 (sm_103a) colour-gradient lattice Boltzmann library with
 * nonorthogonal central moments (Saito, De Rosis, Festuccia, Kaneko, Abe, Koyama,
 * "Color-gradient lattice Boltzmann model with nonorthogonal central moments:
 * Hydrodynamic melt-jet breakup simulations", arXiv:1804.08923).
 *
 * One context holds one D3Q27 lattice resident on one GPU.  lb_step advances it by the
 * paper's time step (Section II): pull streaming with the Section IV.A boundaries, the
 * phase field and its isotropic gradient, the central-moment collision (Eq. (11) with
 * Eqs. (18), (21), (28), (29)), the perturbation (Eq. (30)) and the recolouring
 * (Eqs. (33), (34)).
 *
 * Conventions for every entry point:
 *  - Pointers marked "device" must be CUDA device pointers on the context's device;
 *    "host" pointers are ordinary host memory (pinned memory is faster, not required).
 *  - Every call is ordered on the CUDA stream given at creation.  Only lb_mass, lb_save,
 *    lb_load, the host variants of lb_fields / lb_populations / lb_init, and lb_step at a
 *    check_every boundary synchronise that stream.
 *  - Errors are returned as lb_status; a message for the calling thread is available from
 *    lb_last_error().  No call aborts or throws across this interface.
 *  - Populations are laid out [k][i][z][y][x] (k = 0 red, 1 blue; i in the order of
 *    Eq. (8); x fastest), single precision.
 */
#ifndef LBCM_H
#define LBCM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBCM_ABI_VERSION 2

#if defined(__GNUC__)
#define LB_API __attribute__((visibility("default")))
#else
#define LB_API
#endif

typedef enum {
    LB_OK = 0,
    LB_EINVAL = 1,     /* invalid argument or parameter combination */
    LB_ENOMEM = 2,     /* device allocation failed */
    LB_ECUDA = 3,      /* a CUDA runtime call or kernel launch failed */
    LB_EUNSTABLE = 4,  /* a periodic check found a non-finite colour mass */
    LB_ETIMEOUT = 5,   /* a bounded device wait gave up (the fused step kernel's plane waits) */
    LB_ESTATE = 6,     /* call out of order (e.g. lb_step before lb_init) */
    LB_ENOTIMPL = 7    /* entry point declared but not provided by the library */
} lb_status;

/* Boundary kinds.  z_lo: PERIODIC, FREESLIP or INLET; z_hi: PERIODIC, FREESLIP or CONVECTIVE;
 * PERIODIC must be given for both z ends or neither.  x and y (lb_grid.bc_x, bc_y): PERIODIC
 * or FREESLIP side walls. */
typedef enum {
    LB_BC_PERIODIC = 0,
    LB_BC_FREESLIP = 1,   /* half-way specular reflection (Section IV.A, wall boundaries) */
    LB_BC_INLET = 2,      /* circular inflow disc with free slip around it (Section IV.A) */
    LB_BC_CONVECTIVE = 3  /* first-order implicit convective outflow (Section IV.A) */
} lb_bc;

typedef struct {
    int32_t nx, ny, nz;    /* lattice extent; nx*ny*nz < 2^31 */
    int32_t bc_zlo, bc_zhi;
    int32_t bc_x, bc_y;    /* LB_BC_PERIODIC (0) or LB_BC_FREESLIP side walls (Section IV.A: the
                              jet's side walls are free-slip): a pull whose source lies beyond a
                              wall reads the node's own layer with that velocity component
                              reversed (half-way specular reflection); gradient ghosts mirror
                              the wall layer */
} lb_grid;

/* Population storage.  FP32: every population in single precision.  FP16: the 26 moving
 * populations of each colour are stored in half precision as deviations from the rest
 * equilibrium of the node that will read them (pull streaming), h_i^k = f_i^k -
 * rho_k varphi_i(alpha_k) (Eq. (20)), the rest population in single precision; it takes
 * each colour's remainder of the moving ones as they are read back, so per-node colour mass
 * is kept to FP32 rounding.  FP16_FIT: the same layout, with the deviation taken from a
 * prediction of the reading node, rho_k (1 - alpha-bar) k_q plus an odd part w_i c_i . v_k
 * fitted to the populations it gathered in the step before (v_k kept in FP8 inside the same
 * 16-byte phase entry); about 4x smaller deviations near interfaces, at some extra
 * arithmetic.  Arithmetic is FP32 in all three.  The adjoint needs
 * FP32. */
typedef enum { LB_STORE_FP32 = 0, LB_STORE_FP16 = 1, LB_STORE_FP16_FIT = 2 } lb_storage;

typedef struct {
    double rho_r0, rho_b0;  /* initial densities (Eq. (23)); gamma = rho_r0/rho_b0 >= 19/27 */
    double nu_r, nu_b;      /* kinematic viscosities, > 0; s_2nu from Eq. (16) */
    double sigma;           /* interfacial tension; A = 9 sigma / (4 tau(x)) from Eq. (32) */
    double beta;            /* recolouring parameter of Eqs. (33), (34); 0.7 in the paper */
    double g[3];            /* gravity in the body force F = (rho - rho_b0) g (Eq. (48)) */
    double s0, s1;          /* rates of the conserved moments; 0 in the paper */
    double s2b, s3, s4, s5, s6; /* bulk and higher-order rates; 1 in the paper */
    double u_in;            /* inlet plug velocity u_j0 along +z */
    double d_in;            /* inlet disc diameter D_j0, centred at ((nx-1)/2, (ny-1)/2) */
    double noise_amp;       /* relative amplitude a of the radial inlet noise, 0 = none */
    uint64_t seed;          /* seed of the counter-based inlet noise */
    double eps_grad;        /* regulariser: |grad phi| -> sqrt(|grad phi|^2 + eps^2) */
    int32_t storage;        /* lb_storage */
    int32_t check_every;    /* every so many steps lb_step checks the colour masses (0 = never) */
    double fourier[16];     /* inlet profile u_z = u_in [1 + sum_{m=1..8} (a_m cos m theta + b_m sin m theta)],
                               theta the polar angle of the inlet column about the disc centre;
                               stored a_1, b_1, ..., a_8, b_8 (not in the paper: the parameters the
                               adjoint differentiates); all 0 = the paper's uniform inlet */
    int32_t step_kernel;    /* lb_step with the paper's rates s3..s6 = 1: 0 = one launch per pass
                               (the default, the faster on GB300); 1 = both passes in one cooperative
                               launch of the fused step kernel, whose moments stay in L2 between the
                               passes (less DRAM traffic, more synchronisation).  The same arithmetic,
                               up to the compiler's choice of fused multiply-adds (FP32 rounding) */
    int32_t alpha_mix;      /* alpha-bar of Eqs. (20), (26): 0 = the printed interpolation by
                               (1 +- phi)/2; 1 = by mass fractions rho_k/rho, which makes the
                               equation of state additive over the colours (the reading under
                               which the paper's high-density-ratio droplets stay stable) */
} lb_params;

/* Fills *p with the paper's defaults: rho_r0 = rho_b0 = 1, nu = 1/6, sigma = 0, beta = 0.7,
 * g = 0, s0 = s1 = 0, s2b..s6 = 1, no inlet, eps_grad = 1e-6, FP32 storage, no checks. */
LB_API void lb_params_default(lb_params *p);

typedef struct lb_ctx lb_ctx;

/* Number and byte sizes of the device buffers a context needs (at most LB_MAX_BUFFERS).
 * Buffer 0 and 1: population ping-pong (FP32: 54 * nodes * 4 bytes each; FP16 encodings:
 * 112 bytes per node); 2: order parameter and total density of the step being taken (FP16
 * encodings: one 16-byte phase entry per node and population buffer); 3: outflow history
 * ping-pong; 4: small tables and reduction partials; 5: the collision moments of the step
 * being taken (48 bytes per node: colour densities, mass, momentum and raw second moment,
 * written by the gather pass and read by the collision).  Returns LB_EINVAL for invalid
 * grids or parameters. */
#define LB_MAX_BUFFERS 8
LB_API lb_status lb_buffer_sizes(const lb_grid *grid, const lb_params *params, size_t *sizes_out, int32_t *n_out);

/* Creates a context and allocates its device buffers with cudaMalloc on the current
 * device.  stream: a cudaStream_t (NULL = legacy default stream).  *out is set only on
 * success; the caller releases it with lb_destroy. */
LB_API lb_status lb_create(const lb_grid *grid, const lb_params *params, void *stream, lb_ctx **out);

/* As lb_create, but on caller-owned device memory (e.g. from PyTorch's allocator):
 * bufs[j] must hold at least sizes[j] bytes as reported by lb_buffer_sizes, aligned to
 * 256 bytes.  The buffers must outlive the context; lb_destroy does not free them. */
LB_API lb_status lb_create_with_buffers(const lb_grid *grid, const lb_params *params, void *stream,
                                 void *const *bufs, const size_t *sizes, int32_t n, lb_ctx **out);

/* Initial state kinds for lb_init. */
typedef enum {
    LB_INIT_UNIFORM = 0, /* args = {rho_r, rho_b, ux, uy, uz} */
    LB_INIT_DROPLET = 1, /* args = {R, W}: red sphere of Section III at the domain centre */
    LB_INIT_JET = 2,     /* args unused: quiescent all-blue domain of Section IV.A */
    LB_INIT_FIELDS = 3   /* rho_r, rho_b (nodes each) and u (3*nodes, component-major) given */
} lb_init_kind;

/* Sets populations from fields: f_i^k = rho_k [varphi_i(alpha_k) + w_i (3 cu + 9/2 cu^2
 * - 3/2 u^2 + 9/2 cu^3 - 9/2 cu u^2)] (the equilibrium of Eq. (18) per colour with Phi = 0),
 * copies the outflow plane into the history, and resets the step counter to 0.
 * fields_on_device: 1 if rho_r/rho_b/u are device pointers, 0 for host pointers. */
LB_API lb_status lb_init(lb_ctx *ctx, int32_t kind, const double *args, int32_t nargs,
                  const float *rho_r, const float *rho_b, const float *u, int32_t fields_on_device);

/* Advances the lattice by n >= 0 time steps (Eq. (9) with the operator split of Section II). */
LB_API lb_status lb_step(lb_ctx *ctx, int64_t n);

/* ----------------------------------------------------------- z-slab decomposition
 * One lattice split into slabs of consecutive z planes, one context per slab (on one GPU or
 * several; not in the paper, whose runs are single lattices): the step is a nearest-neighbour
 * stencil, so a slab needs one plane of each neighbour slab per side, twice per step.  A slab's
 * context holds its own planes plus a ghost plane on every side that borders another slab
 * (bc_zlo / bc_zhi of such a side are LB_BC_FREESLIP: the ghost plane computes values that no
 * real plane reads); the first slab keeps the lattice's z_lo boundary, the last its z_hi.
 * One step of the split lattice, on every slab:
 *   1. population halo: lb_halo_pack(LB_HALO_POPULATIONS) of the first and last real plane,
 *      exchanged with the neighbours, lb_halo_unpack into the ghost planes;
 *   2. lb_step_gather: boundary planes and the gather pass (phase field, collision moments);
 *   3. phase halo: the same with LB_HALO_PHASE (the phase entries the gather pass just wrote,
 *      which the collision's gradient stencil and, with FP16 storage, its encoding read);
 *   4. lb_step_collide: the collision; the state advances to t+1.
 * The real planes then evolve bit for bit as the same planes of the whole lattice.  Colour
 * masses of the real planes come from lb_mass_planes, summed over the slabs by the caller.
 *
 * lb_step_gather / lb_step_collide: the two halves of one lb_step (Eq. (9) with the operator
 * split of Section II).  LB_ESTATE for a gather that follows a gather, a collide without a
 * gather, and lb_step or lb_adjoint in between.  Profiling events are not recorded for them.
 * lb_halo_bytes: bytes of one halo plane of the given kind in the context's storage (FP32:
 * 216 (populations) or 8 (phase) per (x, y) column; FP16 encodings: 112 or 16).
 * lb_halo_pack / lb_halo_unpack: copy plane z (0 <= z < nz) of the current populations (kind
 * LB_HALO_POPULATIONS, only outside a split step) or of the phase entries of the step being
 * taken (LB_HALO_PHASE, only between lb_step_gather and lb_step_collide) into / from a
 * contiguous buffer of lb_halo_bytes, in the context's own encoding.  buf is device memory
 * if on_device, else host memory (then the call synchronises).
 * lb_mass_planes: lb_mass restricted to planes [z_begin, z_end).  Synchronises. */
enum { LB_HALO_POPULATIONS = 0, LB_HALO_PHASE = 1 };
LB_API lb_status lb_step_gather(lb_ctx *ctx);
LB_API lb_status lb_step_collide(lb_ctx *ctx);
LB_API lb_status lb_halo_bytes(const lb_ctx *ctx, int32_t kind, size_t *nbytes);
LB_API lb_status lb_halo_pack(lb_ctx *ctx, int32_t kind, int32_t z, void *dst, int32_t on_device);
LB_API lb_status lb_halo_unpack(lb_ctx *ctx, int32_t kind, int32_t z, const void *src, int32_t on_device);
LB_API lb_status lb_mass_planes(lb_ctx *ctx, int32_t z_begin, int32_t z_end, double out[2]);

/* Number of steps taken since lb_init / lb_load. */
LB_API int64_t lb_step_count(const lb_ctx *ctx);

/* Macroscopic fields of the current post-collision state, one float per node each:
 * rho_r, rho_b (sums of the colour populations), phi (Eq. (23)), u_x, u_y, u_z
 * (rho u = sum_i f_i c_i - F/2, the collision having added F), p (Eq. (26) with rho and
 * alpha-bar).  mask selects outputs (bit j = LB_FIELD_*); outs[j] receives field j when
 * its bit is set.  on_device: outs are device (1) or host (0) pointers. */
enum { LB_FIELD_RHO_R = 0, LB_FIELD_RHO_B = 1, LB_FIELD_PHI = 2, LB_FIELD_UX = 3,
       LB_FIELD_UY = 4, LB_FIELD_UZ = 5, LB_FIELD_P = 6, LB_NFIELDS = 7 };
LB_API lb_status lb_fields(lb_ctx *ctx, uint32_t mask, float *const *outs, int32_t on_device);

/* Copies the current populations [k][i][z][y][x] (54 * nodes floats) into out. */
LB_API lb_status lb_populations(lb_ctx *ctx, float *out, int32_t on_device);

/* Copies the outflow history plane [k][i][y][x] (54 * nx * ny floats) into out. */
LB_API lb_status lb_history(lb_ctx *ctx, float *out, int32_t on_device);

/* Per-colour total mass of the current state, summed in FP64 on the device with a
 * fixed-order two-stage reduction (deterministic).  out[0] red, out[1] blue.  A
 * non-finite population makes the corresponding sum non-finite.  Synchronises. */
LB_API lb_status lb_mass(lb_ctx *ctx, double out[2]);

/* Colour masses without any device allocation.  The paper has no counterpart; this is a
 * service for callers that cannot call cudaMalloc: code that keeps its own population
 * arrays under a fixed device-memory budget claimed at start-up (a coupled solver, a
 * process whose memory belongs to another allocator such as PyTorch's) and must not make
 * the driver allocate behind its back, and that has no lb_ctx (whose buffers hold the
 * scratch lb_mass uses).
 *
 * pop: device pointer to populations [2][27][nodes] (FP32, the lb_populations layout) on
 * the current device.  out: device pointer receiving out[0] red, out[1] blue (FP64, the
 * same fixed-order two-stage reduction as lb_mass, with LB_MASS_NOALLOC_CHUNK nodes per
 * first-stage block).  stream: cudaStream_t the work is ordered on; nothing synchronises.
 * nodes must lie in [1, LB_MASS_NOALLOC_MAX_NODES]; larger inputs return LB_EINVAL.
 *
 * The scratch is one file-scope device array of LB_MASS_NOALLOC_SCRATCH_BYTES that every
 * GPU loading the library holds until process exit.  Every call looks up that array's device
 * address (cudaGetSymbolAddress) for the current device and context, so the address stays
 * right after cudaDeviceReset; the first call on a device also loads the library's device
 * code there, so make that first call before any stream capture.  All calls share the array and it
 * keeps the last call's contents; every slot a call reads is written by the same call
 * first, so nothing needs clearing.  Calls whose work overlaps on the GPU (other streams
 * or other host threads) race on the array and must be serialised by the caller. */
#define LB_MASS_NOALLOC_CHUNK 65536
#define LB_MASS_NOALLOC_MAX_BLOCKS 4096
#define LB_MASS_NOALLOC_MAX_NODES ((int64_t)LB_MASS_NOALLOC_CHUNK * LB_MASS_NOALLOC_MAX_BLOCKS)
#define LB_MASS_NOALLOC_SCRATCH_BYTES ((2 * LB_MASS_NOALLOC_MAX_BLOCKS + 2) * 8)
LB_API lb_status lb_mass_noalloc(const float *pop, int64_t nodes, double *out, void *stream);

/* Checkpoint: lb_save writes the state (header, populations, history, step counter) to
 * host memory.  Pass buf = NULL to query the size in *nbytes.  lb_load restores a state
 * saved from a context with the same grid and storage.  Both synchronise. */
LB_API lb_status lb_save(lb_ctx *ctx, void *buf, size_t *nbytes);
LB_API lb_status lb_load(lb_ctx *ctx, const void *buf, size_t nbytes);

/* Kernel timing for profiling.  lb_profile_enable(ctx, capacity) makes the following
 * lb_step calls bracket each kernel launch with CUDA events on the context's stream, for
 * at most `capacity` steps (events are created here, not during stepping); capacity 0
 * disables.  lb_profile_read synchronises, writes per-kernel total device milliseconds
 * and launch counts (index LB_KERNEL_*, up to n_kinds entries), and clears the record. */
/* Index 0 is the boundary planes (one of two kernels, chosen by the plane size); 1 the step's
 * gather pass: moment_kernel with the paper's rates s3..s6 = 1 (phase field and collision
 * moments), phase_field_kernel otherwise; 2 the collision pass; 3 the fused step kernel, which
 * runs both passes in one launch (params.step_kernel = 1). */
enum { LB_KERNEL_BOUNDARY = 0, LB_KERNEL_GATHER = 1, LB_KERNEL_COLLIDE = 2, LB_KERNEL_STEP = 3, LB_NKERNELS = 4,
       LB_KERNEL_PHASE_FIELD = LB_KERNEL_GATHER };
LB_API lb_status lb_profile_enable(lb_ctx *ctx, int32_t capacity);
LB_API lb_status lb_profile_read(lb_ctx *ctx, double *ms, int64_t *launches, int32_t n_kinds);

/* Total number of kernels this context has launched since creation. */
LB_API int64_t lb_kernel_launches(const lb_ctx *ctx);

/* Self-test of a failure path on the device.  which = LB_SELFTEST_FUSED_WAIT runs, on the
 * context's stream, the plane wait of the fused step kernel (params.step_kernel = 1) against a
 * completion target that no gather reaches: the wait gives up after its limit (1 s of the
 * device's global timer), sets the context's error flag and returns, as a wait that ran out
 * inside the fused kernel would.  The call then reads and clears the flag:
 *   *result  LB_ETIMEOUT if the wait gave up and reported it (the expected outcome), else LB_OK
 *   *ms      how long the wait lasted, milliseconds
 * The context's state is untouched and the context stays usable.  Synchronises.  Returns
 * LB_EINVAL for an unknown `which` or NULL outputs, LB_ESTATE inside a split step. */
enum { LB_SELFTEST_FUSED_WAIT = 1 };
LB_API lb_status lb_selftest(lb_ctx *ctx, int32_t which, int32_t *result, double *ms);

/* Replaces the parameters of an existing context (same grid and storage; the state is kept;
 * with FP16 storage rho_r0 and rho_b0 stay fixed once the context holds a state).
 * Validated like lb_create; LB_EINVAL leaves the context unchanged. */
LB_API lb_status lb_set_params(lb_ctx *ctx, const lb_params *params);

/* ---------------------------------------------------------------- discrete adjoint
 * Gradient of an objective J(S(T)) of the state T steps ahead with respect to the inlet
 * velocity u_in, sigma, nu_r, nu_b and the 16 inlet profile coefficients (not in the paper:
 * reverse-mode differentiation of the step of Section II with the boundaries of Section
 * IV.A, transposed by hand).  The forward pass runs T steps from the context's state,
 * keeping a checkpoint every k steps; the reverse pass recomputes each k-step segment from
 * its checkpoint and steps back through it, so device memory holds about T/k + k states.
 * Adjoint arithmetic is FP32, parameter gradients are accumulated in FP64.
 *
 * objective:
 *   LB_OBJ_INTERFACE_AREA  J = sum over nodes with 1 <= z <= nz-2 of sqrt(|grad phi|^2 + eps^2),
 *                          grad phi the isotropic stencil of the order parameter (Eq. (23)) of
 *                          rho_k = sum_i S_i^k; obj_args[0] = eps > 0.
 *   LB_OBJ_PENETRATION     J = delta log sum_n H(phi_n) exp(z_n / delta), H(phi) = ((1 + phi)/2)^2,
 *                          a smooth maximum of z over the red region (H = 1 in pure red, 0 in
 *                          pure blue); obj_args[0] = delta > 0.
 * obj_args[1] and obj_args[3] unused (0); obj_args[2] = checkpoint interval k (0: ceil(sqrt(T))).
 * grad_out (n_grad >= LB_ADJ_NOUT doubles): [0] J, [1] dJ/du_in, [2] dJ/dsigma, [3] dJ/dnu_r,
 *   [4] dJ/dnu_b, [5 + 2(m-1)] dJ/da_m, [6 + 2(m-1)] dJ/db_m for m = 1..8.
 * On return the context holds S(T) (as after lb_step(T)).  Requires FP32 storage and
 * s3 = s4 = s5 = s6 = 1 (LB_EINVAL otherwise); LB_ENOMEM if the workspace cannot be had. */
enum { LB_OBJ_INTERFACE_AREA = 0, LB_OBJ_PENETRATION = 1 };
#define LB_ADJ_NARGS 4
#define LB_ADJ_NOUT 21
LB_API lb_status lb_adjoint(lb_ctx *ctx, int32_t objective, int64_t T, const double *obj_args,
                            double *grad_out, int32_t n_grad);

/* dJ/dS(t0) of the last lb_adjoint, S(t0) the state it started from (the outflow history
 * held fixed), as 54 nx ny nz floats in the canonical layout [k][i][z][y][x].  out is device
 * memory if on_device, else host memory.  LB_ESTATE without a preceding lb_adjoint. */
LB_API lb_status lb_adjoint_state(lb_ctx *ctx, float *out, int32_t on_device);

/* ----------------------------------------------------------------- fragment analysis
 * Fragments of the current state (Section IV.B, diameter procedure): the jet region is
 * phi > 0 (Eq. (23)) of the state's colour densities; fragments are its connected components
 * with face (connectivity 6) or full (26) neighbourhoods, wrapping across periodic boundaries;
 * each has a volume V (nodes) and equivalent spherical diameter d = (6V/pi)^(1/3) (lattice
 * units).  With exclude_inlet on an inlet lattice, components with a node on z = 0 are the
 * continuous column from the nozzle and are left out (their volume is column_volume).  The
 * mass-median diameter is the smallest d at which the fragments with diameter <= d hold at
 * least half of the kept volume (0 without fragments).
 * roots / volumes / diameters (host, each may be NULL): the first min(n_fragments, cap) kept
 * fragments in increasing order of their smallest linear node index (z, y, x row-major), which
 * names them.
 * Device scratch of ~9 B per node is allocated for the call.  LB_EINVAL for connectivity other
 * than 6 or 26. */
typedef struct {
    int64_t n_fragments;          /* kept fragments */
    int64_t column_volume;        /* nodes of the excluded inlet-connected components */
    int64_t total_volume;         /* nodes of the kept fragments */
    double mass_median_diameter;  /* lattice units */
} lb_fragment_stats;
LB_API lb_status lb_fragments(lb_ctx *ctx, int32_t connectivity, int32_t exclude_inlet, int64_t *roots,
                              int64_t *volumes, double *diameters, int64_t cap, lb_fragment_stats *stats);

/* Message for the last failing call made by this thread ("" if none). */
LB_API const char *lb_last_error(void);

/* Releases the context (and its buffers when it allocated them).  NULL is ignored. */
LB_API void lb_destroy(lb_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* LBCM_H */
