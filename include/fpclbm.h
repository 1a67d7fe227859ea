/*
 * fpclbm.h -- C ABI of libfpclbm.so, a GB300 (sm_103a) implementation of the
 * D3Q27 Fokker-Planck central-moment lattice Boltzmann method (FPC-LBM) of
 * Schupbach & Premnath, arXiv 2410.09739.
 *
 * The library advances the distribution functions f_alpha(x, t) of a D3Q27
 * lattice (Sec. 3, "Construction of 3D FPC-LBM") by the collide-and-stream
 * update of Eq. (LBMsteps): per cell, raw moments (Appendix D Step 1), central
 * moments (Step 2), relaxation of every central moment toward its Markovian
 * attractor (Eq. Mvcmattractor3D, Step 3) with body-force sources
 * (Eq. cmupdatesourceD3Q27), back to raw moments and populations (Steps 4, 5)
 * and streaming (Step 6); density and velocity follow Step 7.
 *
 * Conventions shared by every call
 *   - Lattice units: delta_x = delta_t = 1, cs^2 = 1/3 (Sec. 4).
 *   - Field arrays are double, x fastest: idx = x + nx*(y + ny*z).  For an
 *     ensemble the boxes are concatenated in creation order.
 *   - Population arrays are double, alpha-major: f[alpha*N + idx] with alpha
 *     in the order of the paper's velocity list (Sec. 3) and N the cell count.
 *   - Inputs are borrowed for the duration of the call.  Outputs are allocated
 *     by the caller.  "on_device" = 1 means the pointer is a CUDA device
 *     pointer on the handle's device; 0 means host memory (pinned or not).
 *     Page-locked host memory that is mapped into the device's address space
 *     (cudaHostAlloc, cudaHostRegister, pinned framework buffers) is read or
 *     written in place by the field kernels over the host link; other host
 *     memory goes through a device staging buffer.
 *   - The library owns every device allocation it makes; all device work is
 *     ordered on the stream given at creation (NULL = the legacy default
 *     stream).  Calls that return data synchronise that stream; fpclbm_step
 *     synchronises once at its end.
 *   - A handle must not be used by two host threads at once.
 *   - Every call returns an FPCLBM_* status; on failure fpclbm_last_error()
 *     describes it and the handle keeps its previous state unless stated.
 */
#ifndef FPCLBM_H
#define FPCLBM_H

#if defined(__GNUC__)
#define FPCLBM_API __attribute__((visibility("default")))
#else
#define FPCLBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fpclbm* fpclbm_t;

/* Status codes. */
enum {
    FPCLBM_OK = 0,
    FPCLBM_ERR_ARG = -1,      /* bad pointer, size or enum value            */
    FPCLBM_ERR_ALLOC = -2,    /* device or host allocation failed           */
    FPCLBM_ERR_CUDA = -3,     /* a CUDA runtime call failed                 */
    FPCLBM_ERR_PARAM = -4,    /* a relaxation rate outside (0, 2)           */
    FPCLBM_ERR_STATE = -5,    /* e.g. step before init_fields               */
    FPCLBM_ERR_DIVERGED = -6, /* a cell produced rho <= 0, NaN or Inf       */
    FPCLBM_ERR_TIMEOUT = -7   /* a bounded device wait ran out              */
};

/* Arithmetic and storage precision of the populations.  Populations are
 * stored as deviations g = f - w_alpha from the rest state (w = f^eq(1, 0)).
 * FP64: fp64 storage and arithmetic.  FP32: fp32 storage and arithmetic.
 * FP32_STORE_FP16 / FP32_STORE_BF16: fp32 arithmetic, 16-bit storage with
 * round-to-nearest-even. */
enum { FPCLBM_FP64 = 0, FPCLBM_FP32 = 1, FPCLBM_FP32_STORE_FP16 = 2, FPCLBM_FP32_STORE_BF16 = 3 };

/* Boundaries.  PERIODIC: periodic in x, y, z.  WALLS_Y: half-way bounce-back
 * walls at y = -1/2 and y = ny - 1/2 (Sec. 4, cubic cavity), periodic in x
 * and z (channel).  BOX: closed box, half-way bounce-back walls at -1/2 and
 * n - 1/2 on all three axes (the cubic cavity of Sec. 4).  In WALLS_Y and BOX
 * the wall y = ny - 1/2 may move tangentially (fpclbm_set_wall_velocity);
 * every other wall rests.  HALF_CHANNEL: bounce-back wall at y = -1/2 and a
 * specular-reflection symmetry plane at y = ny - 1/2, periodic in x and z
 * (the half channel of the turbulent-channel LES, Sec. 4): a population that
 * leaves the top row along (ex, +1, ez) re-enters it along (ex, -1, ez) at
 * x + (ex, 0, ez). */
enum { FPCLBM_BC_PERIODIC = 0, FPCLBM_BC_WALLS_Y = 1, FPCLBM_BC_BOX = 2, FPCLBM_BC_HALF_CHANNEL = 3 };

/* Choice of the diffusion tensor D' inside the attractors.
 * FP: Eq. (diffusion-tensor-parameter-3D): D' = cs^2 delta for order <= 2 and
 *     D' = kappa~_ij / rho (post-collision second moments) above.
 * EQUILIBRIUM: D' = cs^2 delta at every order with the lower moments at
 *     their own attractors, i.e. Maxwellian central moments (the MCM-LBM the
 *     paper compares with, Sec. 4).
 * FP_LEARNED: FP plus the learned correction of the shear rates installed by
 *     fpclbm_set_closure (no counterpart in the paper); periodic boxes and
 *     channels with resting walls.
 * FP_SMAGORINSKY: FP with the Smagorinsky eddy viscosity and van Driest wall
 *     damping of the turbulent-channel LES (Sec. 4) in the five shear rates,
 *     parameters from fpclbm_set_smagorinsky; boxes with resting walls. */
enum { FPCLBM_DIFF_FP = 0, FPCLBM_DIFF_EQUILIBRIUM = 1, FPCLBM_DIFF_FP_LEARNED = 2, FPCLBM_DIFF_FP_SMAGORINSKY = 3 };

/* Create a single periodic, channel or closed box of nx*ny*nz cells (each >= 1,
 * product < 2^31).  cuda_stream is a cudaStream_t (NULL allowed).
 * Parameters start at tau = 1, drift = 0, diffusion = FP, F = 0; the
 * populations are undefined until fpclbm_init_fields/set_populations.
 * Errors: ARG, ALLOC, CUDA.  *out is NULL on failure. */
FPCLBM_API int fpclbm_create(fpclbm_t* out, int nx, int ny, int nz, int precision, int bc, void* cuda_stream);

/* Create an ensemble of n_boxes independent periodic boxes advanced together
 * by one persistent launch per time step.  dims holds (nx, ny, nz) per box,
 * tau one shear relaxation time per box (see fpclbm_set_params).  Precision
 * FP32 only in this version.  Errors: ARG, PARAM, ALLOC, CUDA. */
FPCLBM_API int fpclbm_create_ensemble(fpclbm_t* out, int n_boxes, const int* dims, const double* tau,
                           int precision, void* cuda_stream);

/* Initialise every cell to the equilibrium of the given density and velocity:
 * f = C(u)^-1 kappa^eq(rho, u), kappa^eq the Maxwellian central moments (the
 * paper gives no initial condition; this is the equilibrium of Sec. 3 at the
 * given fields).  Each stored deviation f - w is that equilibrium rounded
 * once to the storage type (for 16-bit storage after an fp32 evaluation, a few
 * fp32 ulps away).  Resets the step counter to 0.  Errors: ARG, STATE, CUDA. */
FPCLBM_API int fpclbm_init_fields(fpclbm_t h, const double* rho, const double* ux, const double* uy,
                       const double* uz, int on_device);

/* Relaxation parameters.  tau: shear relaxation time; omega_4,5,6,8,9 = 1/tau
 * so that nu = cs^2 (tau - 1/2) (Eq. transportcoeff3DFPCLBM); bulk
 * omega_7 = 1 (zeta = cs^2/3, Sec. 4); omega_0..3 have no effect and are 1.
 * drift = omega_FP: rates of orders k >= 3 are k*omega_FP (Sec. 3,
 * omega_mnp = (m+n+p) omega_FP); drift = 0 selects the paper's experimental
 * choice of unit rates for all orders >= 3 (Sec. 4).  diffusion: FPCLBM_DIFF_*.
 * Every resulting rate must lie in (0, 2), else PARAM and nothing changes.
 * Ensembles: tau scales nothing; per-box tau stays, drift/diffusion apply to
 * all boxes. */
FPCLBM_API int fpclbm_set_params(fpclbm_t h, double tau, double drift, int diffusion);

/* Full override of omega_0..omega_26 in the numbering of Appendix D Step 3:
 * 0:000 1:100 2:010 3:001 4:110 5:101 6:011 7:2s1 8:2d1 9:2d2 10:3s1 11:3m1
 * 12:3s2 13:3m2 14:3s3 15:3m3 16:111 17:4s1 18:4d1 19:4d2 20:211 21:121
 * 22:112 23:122 24:212 25:221 26:222.  Rates 4..26 must lie in (0, 2); 0..3
 * may be any finite value (they cancel).  Single boxes only.  Errors: ARG,
 * PARAM. */
FPCLBM_API int fpclbm_set_rates(fpclbm_t h, const double omega[27]);

/* Constant body force per unit volume (F_x, F_y, F_z), Sec. 3
 * Eq. (forcing:3D); enters as sources sigma_mnp and the half-force velocity
 * of Step 7.  Errors: ARG (non-finite). */
FPCLBM_API int fpclbm_set_force(fpclbm_t h, double Fx, double Fy, double Fz);

/* Smagorinsky subgrid model for FPCLBM_DIFF_FP_SMAGORINSKY (Sec. 4, turbulent
 * channel; the paper names the model, these are its standard definitions):
 * per cell nu_t = (C_s D)^2 |S| (filter width 1), |S| = sqrt(2 S_ij S_ij) with
 * the strain rate from the deviatoric non-equilibrium second-order central
 * moments Pi^d of the incoming populations, S = -Pi^d / (2 rho cs^2 tau), at
 * the effective time tau = tau0 + nu_t / cs^2 (tau0 = 1 / omega_4 of
 * fpclbm_set_params); the closed-form root
 * tau = (tau0 + sqrt(tau0^2 + 18 (C_s D)^2 |Pi^d| / rho)) / 2 sets all five
 * shear rates to 1 / tau.  van Driest damping D = 1 - exp(-y+ / A+),
 * y+ = y_w u* / nu0, y_w the distance of the cell centre to the nearest wall
 * (WALLS_Y: both walls; HALF_CHANNEL: the wall at y = -1/2; PERIODIC: none,
 * D = 1); u* <= 0 or A+ <= 0 switch the damping off.  Defaults 0, 0, 0.
 * Errors: ARG (ensemble, C_s < 0, non-finite). */
FPCLBM_API int fpclbm_set_smagorinsky(fpclbm_t h, double cs, double u_star, double a_plus);

/* Tangential velocity (ux, 0, uz) of the wall y = ny - 1/2 of a WALLS_Y or
 * BOX box (the lid of the lid-driven cavity, Sec. 4; the moving plate of
 * Couette flow).  Half-way bounce-back with the moving-wall momentum
 * correction: a population reflected through that wall is stored as
 * f~_a - 2 w_a rho (e_a . u_w) / cs^2, with w_a the rest weights and rho the
 * density of the fluid cell it leaves; links through the edges and corners of
 * the wall's layer y = ny are corrected too.  Mass is conserved exactly.
 * Starts at 0.  Errors: ARG (periodic box, ensemble, non-finite value). */
FPCLBM_API int fpclbm_set_wall_velocity(fpclbm_t h, double ux, double uz);

/* Advance n >= 0 time steps (collide + stream each).  Replays a captured CUDA
 * graph of the step loop; synchronises the stream once at the end and reads
 * the divergence flag: DIVERGED if any cell saw rho <= 0, NaN or Inf (the
 * populations are then whatever the last step wrote); TIMEOUT if a step
 * kernel's bounded wait for data it staged in shared memory ran out (about a
 * second; that block stored nothing, so the state is not a valid step).
 * Errors: ARG, STATE, CUDA, DIVERGED, TIMEOUT. */
FPCLBM_API int fpclbm_step(fpclbm_t h, long long n);

/* Density and half-force velocity of every cell (Appendix D Step 7:
 * rho = sum f, rho u = sum f e + F/2).  Outputs of N doubles each; any of the
 * four pointers may be NULL to skip it.  The values are the fp64 sums of the
 * stored populations (for fp32 and 16-bit storage formed by compensated fp32
 * summation, equal to the fp64 sums up to their last bits).  Errors: ARG,
 * STATE, CUDA. */
FPCLBM_API int fpclbm_moments(fpclbm_t h, double* rho, double* ux, double* uy, double* uz, int on_device);

/* Global diagnostics reduced in fp64 on the device: out[0] = sum rho,
 * out[1..3] = sum rho u (Step 7 velocity), out[4] = sum rho |u|^2 / 2.
 * Deterministic (fixed reduction order).  out is host memory.
 * Errors: ARG, STATE, CUDA. */
FPCLBM_API int fpclbm_diagnostics(fpclbm_t h, double out[5]);

/* The diagnostics of fpclbm_diagnostics for callers that cannot allocate
 * device memory (no counterpart in the paper).  Some callers must not call
 * cudaMalloc: code embedded in a host application that owns every device
 * allocation through its own pool or arena, or a loop whose latency budget
 * forbids the synchronisation that allocating and freeing imply.  This entry
 * point allocates nothing and needs no handle:
 *   f       device pointer, full populations, double, alpha-major
 *           f[alpha * ncells + cell] in the paper's alpha order (the layout of
 *           fpclbm_get_populations);
 *   ncells  1 .. FPCLBM_NOALLOC_MAX_CELLS, else ARG;
 *   Fx..Fz  body force; the velocity includes half of it, as in
 *           fpclbm_diagnostics;
 *   out     device pointer to 5 doubles: sum rho, sum rho u (3), sum rho|u|^2/2;
 *   cuda_stream  stream to run on (NULL = legacy default stream); the call
 *           does not synchronise it.
 * Its block partials live in a fixed device array inside the library (40 KB
 * on every device that loads it, kept until the process exits).  The first
 * call on a device looks up that array's device address with the device
 * current and caches it: make that first call before any stream capture.
 * The cached address belongs to the device's current primary context: do not
 * use this entry point across a cudaDeviceReset (or anything else that
 * destroys that context) in the same process.
 * Calls share the array; each overwrites the partials it reads, so nothing
 * needs clearing, but calls that overlap on the GPU race -- order them on one
 * stream.  Errors: ARG, CUDA (text via fpclbm_last_error(NULL)). */
#define FPCLBM_NOALLOC_MAX_CELLS 2147483647LL
FPCLBM_API int fpclbm_diagnostics_noalloc(const double* f, long long ncells, double Fx, double Fy, double Fz,
                                          double* out, void* cuda_stream);

/* Copy out / in all populations as full f (not deviations), double,
 * alpha-major in the paper's alpha order, host memory.  get works at any
 * step parity; set leaves the handle at step 0 of a new run.
 * Errors: ARG, STATE (get before init), CUDA. */
FPCLBM_API int fpclbm_get_populations(fpclbm_t h, double* f);
FPCLBM_API int fpclbm_set_populations(fpclbm_t h, const double* f);

/* Populations (full f, double) of the n listed cells only: f[alpha * n + i] for
 * cell index cells[i] (0 <= cells[i] < N), paper alpha order, host memory.
 * For checking single cells of large runs and for probes.  Errors: ARG,
 * STATE, CUDA. */
FPCLBM_API int fpclbm_get_populations_at(fpclbm_t h, const long long* cells, int n, double* f);

/* Steps taken since the last init_fields / set_populations (or the count
 * given to set_state). */
FPCLBM_API int fpclbm_get_step_count(fpclbm_t h, long long* steps);

/* Raw state for bit-identical checkpoint and resume (no counterpart in the
 * paper, which runs no restarts).  get/set_populations go through full fp64
 * populations, which can move the last bit of a stored fp32 or 16-bit
 * deviation; these move the stored deviations themselves, in the storage type
 * and in the library's own layout: for each box in order, 27 slot rows of
 * stride entries (slot s = (ex+1) + 3 (ey+1) + 9 (ez+1), cell x + nx (y + ny z),
 * stride = the box's cell count rounded up to a multiple of 64, the padding
 * entries included), each entry the deviation f - w of the rest state.  Which
 * slot holds which population depends on the AA pattern's parity, i.e. on the
 * step count, which travels with the state.
 *   fpclbm_state_bytes  *bytes = the size of the raw state.
 *   fpclbm_get_state    copies it to raw (host memory of exactly that many
 *                       bytes) and the step count to *steps.  Errors: ARG
 *                       (NULL pointer, wrong size), STATE (before init), CUDA.
 *   fpclbm_set_state    replaces the populations by raw and the step count by
 *                       steps >= 0; the handle is then initialised.  The state
 *                       must come from a handle of the same dimensions,
 *                       precision and boundary kind.  Errors: ARG, CUDA.
 * A resumed run repeats the uninterrupted run bit for bit when the same
 * parameters are set and the same kernel variant runs (the autotuner's choice
 * is cached per process; FPCLBM_TUNE_CACHE or FPCLBM_LAUNCH pin it across
 * processes). */
FPCLBM_API int fpclbm_state_bytes(fpclbm_t h, unsigned long long* bytes);
FPCLBM_API int fpclbm_get_state(fpclbm_t h, void* raw, unsigned long long bytes, long long* steps);
FPCLBM_API int fpclbm_set_state(fpclbm_t h, const void* raw, unsigned long long bytes, long long steps);

/* Test hook (no counterpart in the paper): every device and page-locked host
 * allocation of the library's handles and training scratch goes through one
 * wrapper that counts live allocations.  fail_after >= 0 makes the allocation
 * that follows fail_after further successful ones fail as if the device were
 * out of memory (once); -1 disarms; other values leave the setting as it is.
 * *live (if not NULL) receives the number of live allocations, so a test can
 * check that a failed call freed everything it had allocated.  Returns OK. */
FPCLBM_API int fpclbm_test_alloc_hook(int fail_after, long long* live);

/* Launch configuration of the step kernel, for reports (no counterpart in the
 * paper: it names which of the library's equivalent kernels runs).  Valid after
 * the first fpclbm_step since the last change of parameters, force or wall
 * velocity (the autotuner chooses then); before that FPCLBM_ERR_STATE.
 * out[0] threads per block; out[1] register-cap class (resident blocks of the
 * one-cell kernel: 1 none, 2 ~128, 3 ~80, 4 64 registers), or for variant 3
 * its number of shared-memory stages; out[2] variant (0 one cell per thread,
 * 1 cp.async-pipelined, 2 two cells per thread on the packed fp32 pipe, 3 two
 * cells per thread with whole slot rows moved through shared memory by bulk
 * asynchronous copies; ensembles: 0 or 2); out[3] collision mode (0 FP, 1 MCM,
 * 2 FP + learned closure, 3 FP + Smagorinsky, 4 FP, 5 MCM and 6 FP + learned
 * closure with every rate of orders 3-6 equal to 1, where those moments are set
 * to their attractors plus half their body-force sources).  out is
 * caller-owned int[4]. */
FPCLBM_API int fpclbm_get_launch(fpclbm_t h, int out[4]);

/* The learned closure's weights in the device layout the fused inference reads
 * (no counterpart in the paper; the layout test of the host packing runs it
 * without a GPU).  w: the 4865 bf16 bit patterns of fpclbm_set_closure, in
 * its order; out: caller-owned, out_words = 3012 32-bit words: [0, 512) the
 * layer-1 B fragments of mma.sync.m16n8k16 per (n-tile nt, lane): words
 * (nt * 32 + lane) * 2 + {0, 1}, each two bf16 of consecutive k (lower k in the
 * low half), k = 2t, 2t+1 and 2t+8, 2t+9 for lane = 4g + t, output n = 8 nt + g,
 * with b1 at k = 9; [512, 2560) the layer-2 B fragments, words
 * ((nt * 4 + kt) * 32 + lane) * 2 + {0, 1}, k = 16 kt + the same offsets;
 * [2560, 2624) b1, [2624, 2688) b2, [2688, 2752) W3 and [2752] b3 as fp32 bit
 * patterns; [2756, 3012) per (nt, lane) the bf16 of b2[8 nt + g] for t = 0,
 * else 0 (the first word of a B fragment whose only non-zero K row is 64).
 * Pure host code.  Errors: ARG for a NULL pointer or other sizes. */
FPCLBM_API int fpclbm_closure_pack(const unsigned short* w, int n_params, unsigned int* out, int out_words);

/* Install the learned closure used by FPCLBM_DIFF_FP_LEARNED: a per-cell
 * MLP 9 -> 64 -> 64 -> 1 (tanh hidden layers) whose inputs are the six
 * non-equilibrium second-order central moments and u, and whose output
 * delta omega corrects the shear rates omega_4,5,6,8,9 of the cell to
 * max(omega + min(delta omega, 0), 0.02): the correction only adds viscosity,
 * as the eddy-viscosity labels it is trained on do.  Weights are
 * bf16 bit patterns, n_params = 4865, in the order W1[64][9], b1[64],
 * W2[64][64], b2[64], W3[1][64], b3[1] (row-major, out x in).  No
 * counterpart in the paper, whose channel uses a Smagorinsky LES (Sec. 4).
 * Errors: ARG. */
FPCLBM_API int fpclbm_set_closure(fpclbm_t h, const unsigned short* bf16_weights, int n_params);

/* Training data for the learned closure from a fine single box (no
 * counterpart in the paper).  The box is cut into r x r x r blocks ("coarse
 * cells", x fastest; nx, ny, nz multiples of r; ny / r >= 2 with walls).  Per
 * coarse cell c it writes 9 features X[9 c + k] and a label T[c] (float;
 * device pointers when on_device = 1, else host):
 *   features  the non-equilibrium second-order central moments that a coarse
 *             FPC-LBM with shear relaxation time tau_coarse carries for the
 *             filtered flow, -2 rho cs^2 tau_coarse S_ij for ij = xx, yy, zz,
 *             xy, xz, yz (Appendix C, Eq. noneqmmoments3D, with the discrete
 *             1/omega -> tau), followed by the filtered velocity (3);
 *   label     the shear-rate change that adds the sub-filter eddy viscosity:
 *             1/((nu + nu_t)/cs^2 + 1/2) - 1/(nu/cs^2 + 1/2),
 *             nu = cs^2 (tau_coarse - 1/2) (Eq. transportcoeff3DFPCLBM),
 *             nu_t = max(0, -tau^d_ij S_ij / (2 S_kl S_kl)),
 *             tau_ij = <u_i u_j> - <u_i><u_j>.
 * <.> is the plain mean over the r^3 fine cells (rho, Step 7 velocity u,
 * u_i u_j); S_ij is the strain rate of <u> by central differences in coarse
 * cells (periodic in x, z; next to a y wall the derivative of the quadratic
 * through the no-slip wall value 0 at y = -1/2 or ny/r - 1/2 and the two
 * nearest rows: <u>_0 + <u>_1 / 3 at the first row).  Lattice velocities are
 * unchanged under acoustic scaling (dt/dx fixed), so features and labels are
 * in coarse lattice units.  Errors: ARG, STATE, ALLOC, CUDA. */
FPCLBM_API int fpclbm_closure_sample(fpclbm_t fine, int r, double tau_coarse, float* X, float* T, int on_device);

/* Train the closure network (layout of fpclbm_set_closure) on n samples,
 * device arrays X[n][9] and T[n], by Adam (learning rate lr, beta 0.9/0.999)
 * on the mean squared error for `epochs` passes in mini-batches of `batch`,
 * each epoch in a fresh pseudo-random order; initial weights are drawn from
 * `seed`.  Inputs and target are standardised during training; the weights
 * written to out_bf16 (4865 bf16 bit patterns, host) have the
 * standardisation folded into W1, b1, W3, b3, so fpclbm_set_closure applies
 * them to raw inputs.  The forward and backward kernels use the bf16 weights
 * with fp32 accumulation; fp32 master weights and gradients; the loss is
 * accumulated in fp64.  loss_per_epoch (host, may be NULL) receives each
 * epoch's mean squared error in standardised units.  Allocates its own
 * device buffers for the call.  No counterpart in the paper.
 * Errors: ARG, ALLOC, CUDA (text via fpclbm_last_error(NULL)). */
FPCLBM_API int fpclbm_closure_train(const float* X, const float* T, long long n, int epochs, int batch, double lr,
                                    unsigned long long seed, unsigned short* out_bf16, double* loss_per_epoch,
                                    void* cuda_stream);

/* One evaluation of the closure network's mean squared error on n samples
 * (device arrays X[n][9], T[n], raw units) with the given bf16 weights (host):
 * loss (host, fp64) and its gradient (host, 4865 fp32 values in the weight
 * layout), computed by the training kernels.  For checking them against an
 * fp64 reference.  Errors: ARG, ALLOC, CUDA. */
FPCLBM_API int fpclbm_closure_grad(const float* X, const float* T, int n, const unsigned short* bf16_weights,
                                   float* grad, double* loss, void* cuda_stream);

/* Release everything the handle owns.  NULL is a no-op.  Returns OK. */
FPCLBM_API int fpclbm_destroy(fpclbm_t h);

/* Text of the last error on this handle ("" if none); owned by the handle
 * and valid until its next call.  With h = NULL: the last error of a failed
 * fpclbm_create / fpclbm_create_ensemble on this thread. */
FPCLBM_API const char* fpclbm_last_error(fpclbm_t h);

/* ------------------------------------------------------------------------ */
/* The 2D FPC-LBM on the D2Q9 lattice (Sec. 2 and the appendix on the 2D     */
/* algorithm).  A separate handle: nx x ny boxes (periodic or closed), populations in the */
/* velocity order of Sec. 2 (e_x = 0,1,0,-1,0,1,-1,-1,1; e_y = 0,0,1,0,-1,1, */
/* 1,-1,-1), stored as deviations from the rest weights (4/9, 1/9, 1/36) in  */
/* the given precision, AA-pattern update in place.  Rates omega_0..omega_8  */
/* in the 2D Step 3 numbering: 3 = 2s (bulk, zeta = cs^2 (1/omega_3 - 1/2)), */
/* 4 = 2d and 5 = 11 (shear, nu = cs^2 (1/omega_4 - 1/2)), 6 = 21, 7 = 12,   */
/* 8 = 22 (Eq. transportcoeff2DFPCLBM).  Return codes as above.              */
/* ------------------------------------------------------------------------ */
typedef struct fpclbm2d* fpclbm2d_t;

/* Periodic nx x ny box (nx, ny >= 1, nx * ny < 2^31), any FPCLBM_* precision.
 * Starts at tau = 1, unit rates, no force, FP mode.  Errors: ARG, ALLOC. */
FPCLBM_API int fpclbm2d_create(fpclbm2d_t* out, int nx, int ny, int precision, void* cuda_stream);

/* Equilibrium of (rho, ux, uy) per cell (x fastest), f = C(u)^-1 kappa^eq with
 * the Maxwellian central moments; resets the step count.  on_device: the
 * three arrays are device pointers.  Errors: ARG, CUDA. */
FPCLBM_API int fpclbm2d_init_fields(fpclbm2d_t h, const double* rho, const double* ux, const double* uy,
                                    int on_device);

/* omega_4 = omega_5 = 1/tau; omega_3 = bulk_rate (0 selects 1); orders 3 and 4:
 * order * drift when drift > 0, else 1 (as in 3D); diffusion: FPCLBM_DIFF_FP or
 * FPCLBM_DIFF_EQUILIBRIUM (MCM).  Rates 3..8 must lie in (0, 2), else PARAM.
 * Errors: ARG, PARAM. */
FPCLBM_API int fpclbm2d_set_params(fpclbm2d_t h, double tau, double bulk_rate, double drift, int diffusion);

/* Full override of omega_0..omega_8 (0..2 have no effect).  Errors: ARG, PARAM. */
FPCLBM_API int fpclbm2d_set_rates(fpclbm2d_t h, const double omega[9]);

/* Body force (Eq. forcing:2D).  Errors: ARG. */
FPCLBM_API int fpclbm2d_set_force(fpclbm2d_t h, double Fx, double Fy);

/* Boundary of the 2D box: FPCLBM_BC_PERIODIC (default) or FPCLBM_BC_BOX, a
 * closed square box with half-way bounce-back at -1/2 and n - 1/2 on both
 * axes whose wall y = ny - 1/2 moves along x at lid_ux (the 2D lid-driven
 * cavity of Sec. 4; momentum-corrected as in fpclbm_set_wall_velocity).
 * lid_ux must be 0 for PERIODIC.  Changing the boundary is allowed at even
 * step counts only (the AA layout of the odd parity depends on it).
 * Errors: ARG, STATE. */
FPCLBM_API int fpclbm2d_set_boundary(fpclbm2d_t h, int bc, double lid_ux);

/* Advance n >= 0 steps; DIVERGED if a cell saw rho <= 0 or a non-finite value.
 * Errors: ARG, STATE, CUDA, DIVERGED. */
FPCLBM_API int fpclbm2d_step(fpclbm2d_t h, long long n);

/* rho and the half-force velocity per cell (any pointer may be NULL).
 * Errors: ARG, STATE, CUDA. */
FPCLBM_API int fpclbm2d_moments(fpclbm2d_t h, double* rho, double* ux, double* uy, int on_device);

/* Full populations f[alpha * N + cell] (host, 9 N doubles), in and out;
 * setting them resets the step count.  Errors: ARG, STATE, CUDA. */
FPCLBM_API int fpclbm2d_get_populations(fpclbm2d_t h, double* f);
FPCLBM_API int fpclbm2d_set_populations(fpclbm2d_t h, const double* f);

/* NULL-safe. */
FPCLBM_API int fpclbm2d_destroy(fpclbm2d_t h);

/* Message of the last failed call on h (or of the last failed create when h
 * is NULL); owned by the library, valid until the next call. */
FPCLBM_API const char* fpclbm2d_last_error(fpclbm2d_t h);

#ifdef __cplusplus
}
#endif
#endif /* FPCLBM_H */
