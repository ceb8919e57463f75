/* dgfs.h -- C ABI of the GB300 fast Fourier spectral collision library.
 *
 * The library evaluates the multi-species Boltzmann collision operator
 *
 *     Q_ij(f_i, f_j)(v) = int_{R^3} int_{S^2} B_ij [ f_i(v') f_j(v_*') - f_i(v) f_j(v_*) ] dsigma dv_*
 *
 * (Sec. 2; nondimensional form Eq. NMCO, kernel Eq. NVSS) for every ordered species pair
 * (i, j) at every node of a batch, by the fast Fourier spectral method of Sec. 4:
 * truncated Fourier series on [-L, L]^3 with N^3 modes, the gain weight split of Eq. GG
 * evaluated with an N_rho-point Gauss-Legendre rule in rho and an M-point spherical design in
 * sigma (each (rho, sigma) term is a product of two phase-shifted inverse transforms taken
 * through a forward transform), and the loss term as the convolution of f_i with G^- f_j.
 * Every DG node is an independent evaluation (Sec. 5.1: the nodal GLL basis makes the
 * collision tensor diagonal), so a batch is a list of nodes.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid      : N points per axis, cell-centred, v_n = -L + (n + 1/2) 2L/N.  Q at the grid
 *             points depends only on the sampled values of f, not on this offset.
 * Layouts   : f[batch][s][N][N][N] and Q[batch][s][s][N][N][N] (x slowest, z fastest),
 *             Q[b][i][j] = Q_ij(f_i, f_j) at node b.  Element type: double for DGFS_FP64
 *             plans, float for DGFS_FP32 and DGFS_BF16X3 plans.
 * Ownership : the caller owns f and Q.  f is only read; every element of Q is written.
 *             The plan owns its tables and its workspace (device memory on the device that
 *             was current at dgfs_create_plan).
 * Streams   : device entry points are asynchronous and ordered on the given cudaStream_t
 *             (NULL = legacy default stream); they never synchronise the device.
 * Threads   : a plan is not thread-safe; distinct plans may run concurrently on distinct
 *             streams.  Evaluations of one plan use its single workspace: one enqueued on a
 *             different stream than the plan's previous evaluation first waits for that
 *             evaluation (cudaStreamWaitEvent), so they never overlap on the device.  An
 *             evaluation recorded into a CUDA graph (stream capture) is ordered by the graph
 *             instead: the caller keeps replays of that graph from overlapping other
 *             evaluations of the plan, and keeps the plan alive while the graph is used.
 * Errors    : 0 on success, a negative DGFS_ERR_* code otherwise; dgfs_strerror() names it.
 *             Arguments are checked before any work is enqueued.
 */
#ifndef DGFS_H
#define DGFS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define DGFS_OK 0
#define DGFS_ERR_INVALID_ARG (-1)    /* a NULL pointer, a size or a parameter out of range */
#define DGFS_ERR_UNSUPPORTED_N (-2)  /* N is not one of 4, 6, 8, 12, 16, 24, 32, 48 */
#define DGFS_ERR_OOM (-3)            /* device or host allocation failed */
#define DGFS_ERR_BUDGET (-4)         /* batch larger than the plan's max_batch */
#define DGFS_ERR_CUDA (-5)           /* a CUDA runtime call or kernel launch failed */
#define DGFS_ERR_DEVICE_TIMEOUT (-6) /* a bounded device-side wait gave up: the DGFS_BF16X3
                                        kernel waits at most about one second for each batch
                                        of its tensor-core MMAs, the FP32 collision kernel
                                        (N = 24, 48) for each staged plane copy, then they
                                        stop and record it; reported by dgfs_plan_check and
                                        dgfs_dft3_bf16x3 */
#define DGFS_ERR_UNSUPPORTED (-7)    /* a valid request this build does not implement */

/* arithmetic of the transforms, products and accumulations */
#define DGFS_FP64 0
#define DGFS_FP32 1
#define DGFS_BF16X3 2 /* the transforms as dense matrix products on the tensor cores: every FP32
                         operand split exactly into three BF16 terms, the six products of order
                         down to 2^-16 accumulated in FP32 (f and Q in float, like DGFS_FP32).
                         VHS only (alpha = 1), N in {8, 16, 24}; else DGFS_ERR_UNSUPPORTED or
                         DGFS_ERR_UNSUPPORTED_N at plan creation */

/* plan flags */
#define DGFS_CONSERVE 1u    /* project each self pair and each stacked cross pair onto the
                               discrete conservation laws (Eq. consv) with FP64 moment sums */
#define DGFS_SUM_SPECIES 2u /* return sum_j kappa_ij Q_ij per species (Eq. NMBE right-hand side) */
#define DGFS_PER_PAIR_R 8u  /* each ordered pair (i, j) gets its own radial truncation
                               R_ij = 2 S_ij, S_ij the support Eq. domain allows for that pair
                               alone, with its own N_rho-point rule, instead of the common
                               R = 2 min S_ij (requires R <= 0 in the description; the (i,j)
                               and (j,i) products are then not shared) */
#define DGFS_LOSS_ACCURATE 4u /* radial integral of the loss weight G^- (defined after Eq. GG)
                                 with its own 4 N_rho-point Gauss-Legendre rule on [0, R]
                                 instead of the gain's N_rho nodes (the paper only asks for
                                 G^- "to high accuracy") */

typedef struct dgfs_plan_s* dgfs_plan; /* opaque, owned by the library */

/* Plan description.  All arrays are host memory, read during dgfs_create_plan only. */
typedef struct {
  int N;                   /* grid points per axis, one of 4, 6, 8, 12, 16, 24, 32, 48 */
  double L;                /* half width of the velocity domain [-L, L]^3 (Sec. 4), > 0 */
  int s;                   /* number of species, 1..8 */
  const double* mass;      /* [s] nondimensional masses m_i / m_0 (Sec. 3), > 0 */
  const double* omega;     /* [s*s] row-major (i, j): viscosity index omega_ij in [0.5, 1] */
  const double* alpha;     /* [s*s]: VSS scattering parameter alpha_ij in [1, 2]; 1 = VHS.  Any
                              alpha != 1 selects the sigma-dependent complex gain table
                              [s*s][N_rho][slots][N^3], one slot per direction without an
                              antipode and per antipodal pair (M / 2 slots for an antipodal
                              rule, since F(-sigma) = conj F(sigma)) */
  const double* b_override;/* nullable [s*s]: kernel prefactor b_ij replacing Eq. NVSS */
  int M;                   /* sphere points; with sigma == NULL one of 6, 12, 32 */
  const double* sigma;     /* nullable [M*3]: unit directions of the sphere rule */
  const double* w_sigma;   /* nullable [M]: its weights (default 4 pi / M each) */
  int N_rho;               /* Gauss-Legendre points in rho on [0, R], >= 1 */
  double R;                /* radial truncation; <= 0 selects R = 2S with S from Eq. domain */
  int precision;           /* DGFS_FP64, DGFS_FP32 or DGFS_BF16X3 */
  unsigned flags;          /* 0 or DGFS_CONSERVE | DGFS_SUM_SPECIES | DGFS_LOSS_ACCURATE |
                              DGFS_PER_PAIR_R */
  int max_batch;           /* largest batch of a host-buffer call or of a DGFS_SUM_SPECIES plan */
  const double* kappa;     /* nullable [s*s]: species-sum weights kappa_ij (e.g. 1/Kn_ij, Eq. Kn);
                              NULL = 1.  Used with DGFS_SUM_SPECIES only. */
} dgfs_plan_desc;

/* Build the tables (Gauss-Legendre rule, design, b_ij of Eq. NVSS, R of Eq. domain, gain
 * weights F^(ij)(k, rho) of Eq. GG and loss weights G^(ij)-(k), computed in FP64, the
 * N^3-sized ones on the device; a DGFS_FP32 plan keeps them rounded once to FP32) and the
 * workspace on the current device.  *out receives the plan.  Device memory is allocated
 * stream-ordered on a stream the plan owns; the call returns when the plan is ready and
 * never synchronises other streams.  Errors, before any device work: DGFS_ERR_UNSUPPORTED_N
 * for N outside the list of the N field; DGFS_ERR_INVALID_ARG for a field outside its stated range,
 * a non-finite mass, b_ij, kappa, weight or R, a direction that is not a unit vector, an
 * unknown flag, or R > 0 with DGFS_PER_PAIR_R.  DGFS_ERR_OOM when the tables or the
 * workspace do not fit.  DGFS_ERR_CUDA when a CUDA call fails, or when the collision kernel
 * of a shape that keeps its accumulators in tensor memory (FP32, N = 32) could be placed
 * more times per SM than the SM's 512 tensor-memory columns allow (judged from the built
 * kernel's registers and shared memory; such a CTA would wait inside its cluster). */
int dgfs_create_plan(const dgfs_plan_desc* desc, dgfs_plan* out);

/* Release the plan's device memory.  Waits for the plan's most recent evaluation (not for
 * the rest of the device) and frees stream-ordered. */
int dgfs_destroy_plan(dgfs_plan plan);

/* Q = all s^2 collision operators of the batch (Sec. 4), device pointers, stream-ordered.
 * f_dev: [batch][s][N][N][N], Q_dev: [batch][s][s][N][N][N], element type per precision,
 * both 16-byte aligned.  batch >= 0 (0 is a no-op).  Calls on one plan share its workspace:
 * the library orders a call issued on another stream after the plan's previous one (see
 * Threads above).
 * With DGFS_CONSERVE every self pair Q_ii and every stacked cross pair [Q_ij; Q_ji] is
 * replaced by its nearest (L2) vector satisfying the discrete laws of Eq. consv: mass of each
 * operator, and m_i w_ij int v Q_ij + m_j w_ji int v Q_ji = 0 and the same with |v|^2, with
 * w_ij = 1 / b_ij (the pair weights under which the kernel is symmetric, b_ij kappa = 1/Kn_ij
 * for Eq. NVSS); the moment sums and the 5x5 / 6x6 solves are FP64 on the device.
 * With DGFS_SUM_SPECIES Q_dev is [batch][s][N][N][N] and receives sum_j kappa_ij Q_ij; then
 * batch <= max_batch (else DGFS_ERR_BUDGET), the full operators being staged in the plan. */
int dgfs_eval_collision(dgfs_plan plan, const void* f_dev, void* Q_dev, int batch, void* stream);

/* The same evaluation from host buffers (pinned or pageable; pinned lets the copies run
 * asynchronously): copies f to the device, evaluates, copies Q back and returns when Q is in
 * host memory.  Batches of 512 nodes or more are split into up to 8 chunks whose input copy,
 * evaluation and output copy (on two copy streams the plan owns) overlap; the chunks'
 * evaluations alternate between `stream` and a second stream of the plan, each with a
 * workspace of its own, so one chunk's kernel starts while the previous one ends.  The call
 * is ordered after the work already on `stream` and after the plan's previous evaluation.
 * batch <= max_batch, else DGFS_ERR_BUDGET.  The plan's staging buffers and second workspace
 * are allocated at the first call. */
int dgfs_eval_collision_host(dgfs_plan plan, const void* f_host, void* Q_host, int batch,
                             void* stream);

/* Device bytes of the plan's tables and workspace (with batch > 0 the workspace includes what
 * a host-buffer call of `batch` nodes adds: staging and the second workspace). */
int dgfs_plan_bytes(dgfs_plan plan, int batch, size_t* tables, size_t* workspace);

/* The radial truncation R the plan uses (R = 2S from Eq. domain unless given; with
 * DGFS_PER_PAIR_R the common R, the pairs using their own R_ij = 2 S_ij >= R). */
int dgfs_plan_radius(dgfs_plan plan, double* R);

/* One step of the second-order strong-stability-preserving Runge-Kutta scheme (the time
 * integrator of Sec. 5, used with dt = 0.01 for the Krook-Wu evolution of Sec. 6.1) for the
 * spatially homogeneous equation d_t f_i = sum_j kappa_ij Q_ij(f_i, f_j), in place on f_dev
 * [batch][s][N][N][N]:  f1 = f + dt R(f);  f <- (f + f1 + dt R(f1)) / 2, R being the plan's
 * species-summed operator.  Needs a DGFS_SUM_SPECIES plan (DGFS_CONSERVE applies to each
 * evaluation if set) and batch <= max_batch; the two work arrays are allocated at the first
 * call.  Stream-ordered, asynchronous. */
int dgfs_ssp_rk2_step(dgfs_plan plan, void* f_dev, double dt, int batch, void* stream);

/* Limit one launch of the persistent collision kernel to a fraction 0 < share <= 1 of the
 * thread-block clusters the device holds (default 1).  Evaluations of different plans on
 * different streams then share the SMs instead of queueing behind one another (serving). */
int dgfs_plan_set_sm_share(dgfs_plan plan, double share);

/* Workspace integrity check (a stand-in for a memory checker): the plan's workspace lies
 * between two 4 KB guard blocks of a fixed byte pattern written at plan creation.  After the
 * plan's most recent evaluation (waited for on the plan's own stream; evaluations recorded
 * into a CUDA graph must have completed before the call), both blocks are read back and
 * *intact = 1 when every byte still holds the pattern, 0 when a kernel wrote outside the
 * workspace.  Returns DGFS_ERR_DEVICE_TIMEOUT (with *intact set) when a kernel of the plan
 * recorded that one of its bounded device-side waits gave up.  Errors: DGFS_ERR_INVALID_ARG
 * (null plan or pointer), DGFS_ERR_CUDA. */
int dgfs_plan_check(dgfs_plan plan, int* intact);

/* Kernels enqueued by the most recent evaluation on this plan. */
int dgfs_plan_launches(dgfs_plan plan, int* launches);

/* Static text naming a return code. */
const char* dgfs_strerror(int code);

/* Batched 3D discrete Fourier transform on the tensor cores, the building block of the
 * DGFS_BF16X3 path (the truncated Fourier series of Sec. 4 and its coefficients are such
 * transforms on the N^3 grid):  y_v[n] = sum_k x_v[k] e^{dir 2 pi i k.n / N}, unnormalised,
 * for v = 0..count-1.  x_dev and y_dev: [count][N][N][N] complex float (interleaved re, im),
 * device memory, 16-byte aligned, not overlapping; N in {8, 16, 24} (else
 * DGFS_ERR_UNSUPPORTED_N); dir = -1 (forward) or +1 (inverse), else DGFS_ERR_INVALID_ARG.  Each
 * axis is one pass of tensor-core matrix products with every FP32 operand split into three BF16
 * terms (as DGFS_BF16X3).  Allocates a 14 KB matrix image stream-ordered on `stream`, runs, and
 * returns when done (synchronises `stream`); DGFS_ERR_DEVICE_TIMEOUT when the kernel's bounded
 * wait for its MMAs gave up. */
int dgfs_dft3_bf16x3(int N, int dir, const void* x_dev, void* y_dev, int count, void* stream);

/* Self-check of the bounded device-side wait that the DGFS_BF16X3 kernels use for their MMAs
 * and bulk copies (no counterpart in the paper; failure detection).  One CTA waits on an
 * mbarrier that nothing completes, giving up after `seconds` (0 < seconds <= 10) of SM clock
 * at the device's reported clock rate.  Returns DGFS_ERR_DEVICE_TIMEOUT when the wait gave up
 * and reported it, as designed, and leaves the context usable; DGFS_OK would mean the wait
 * returned without the barrier completing.  Synchronous; allocates 4 bytes.  Errors:
 * DGFS_ERR_INVALID_ARG, DGFS_ERR_OOM, DGFS_ERR_CUDA. */
int dgfs_check_bounded_wait(double seconds);

/* Measured multiply-add rate of the current device's FP32 (precision = DGFS_FP32) or FP64
 * (DGFS_FP64) pipe, in flop/s (2 flop per FMA): the denominator of the ALU roofline that bounds
 * the collision kernel.  No counterpart in the paper (a measurement helper).  Runs a
 * dependent-FMA loop on every SM for about 50 ms after two sizing launches, on the legacy
 * default stream, and returns when done (synchronous; allocates and frees a small output
 * buffer).  The rate is that of the SM clock during the call.  Errors: DGFS_ERR_INVALID_ARG
 * (null pointer, other precision), DGFS_ERR_OOM, DGFS_ERR_CUDA. */
int dgfs_measure_fma_rate(int precision, double* flop_per_s);

/* The evaluation of dgfs_eval_collision for callers that cannot allocate device memory
 * (no counterpart in the paper; it exists for embedding).  A solver plugin whose host
 * application owns every device allocation, or code that may not call cudaMalloc after
 * start-up, cannot create a plan, because dgfs_create_plan allocates tables and a workspace.
 * This call takes the plan description itself, needs no plan, and allocates nothing: the
 * quadrature and kernel constants travel in the kernel's parameter block, the gain and loss
 * weights and the phase factors are computed inside the kernel, and the workspace is a
 * static device array of 14.7 MB (64 work slots of 7 * 16^3 complex floats) that every GPU
 * loading the library holds until the process exits.
 *
 * desc, f_dev, Q_dev, batch and stream mean what they mean for dgfs_create_plan and
 * dgfs_eval_collision (f and Q on the current device, float, 16-byte aligned);
 * desc->max_batch is ignored.  Limits: desc->precision == DGFS_FP32, N in {8, 12, 16}
 * (else DGFS_ERR_UNSUPPORTED_N), s <= 3, M <= 12, N_rho <= 16, alpha == 1 (else
 * DGFS_ERR_UNSUPPORTED); these are checked before any work.  Batches of any size run on at
 * most 64 CTAs.
 * The first call in a CUDA context (per device, and again after cudaDeviceReset or any other
 * change of the device's current context) looks up the workspace's device address and sets
 * the kernels' shared-memory limits (cudaGetSymbolAddress, cudaFuncSetAttribute); make that
 * first call before any stream capture.  desc fields must be finite (L, R, b_override,
 * w_sigma, sigma), else DGFS_ERR_INVALID_ARG.  Every call on a device shares the one workspace: calls whose
 * kernels overlap on the GPU (different streams, no ordering between them) race and give
 * wrong results; calls ordered on one stream do not.  Results equal dgfs_eval_collision's
 * within FP32 rounding. */
int dgfs_eval_collision_noalloc(const dgfs_plan_desc* desc, const void* f_dev, void* Q_dev,
                                int batch, void* stream);

/* ---------------------------------------------------------------------------------------
 * One-dimensional nodal DG in physical space (Sec. 5): the spatially inhomogeneous equation
 * d_t f_i + v_x d_x f_i = sum_j kappa_ij Q_ij(f_i, f_j) (Eq. NMBE, kappa_ij = 1/Kn_ij) on
 * [x0, x1], split into Ne equal elements, each carrying K Gauss-Lobatto-Legendre nodes with
 * the Lagrange basis on them.  As in Sec. 5 the mass matrix and the collision tensor are taken
 * with the GLL rule, so both are diagonal and the collision term is the species-summed
 * operator at every node; the stiffness matrix is exact; the face flux is upwind; the time
 * step is SSP-RK2.  Walls take the Maxwell boundary condition of Sec. 2, with the wall
 * density n_w from zero net mass flux through the wall, evaluated as sums over the
 * velocity grid.
 *
 * State layout: f[Ne][K][s][N][N][N] (element, node, species, velocity grid as for
 * dgfs_eval_collision), i.e. batch = Ne * K collision nodes, element type of the collision
 * plan's precision, device memory, 16-byte aligned, owned by the caller.  Node positions come
 * from dgfs_dg_nodes. */
typedef struct dgfs_dg_plan_s* dgfs_dg_plan; /* opaque, owned by the library */

#define DGFS_BC_PERIODIC 0 /* f(x1) continues at x0 */
#define DGFS_BC_WALLS 1    /* boundary sides at x0 (outward normal -x) and x1 (+x), each a
                              Maxwell wall or an in-flow boundary (side[]) */
#define DGFS_SIDE_WALL 0   /* Maxwell wall condition (Sec. 2) */
#define DGFS_SIDE_INFLOW 1 /* in-flow equilibrium condition (Sec. 2): entering particles of
                              species i follow n_in_i (m_i / (pi T))^(3/2) exp(-m_i |v - u|^2 / T) */

typedef struct {
  int Ne;          /* elements, >= 1 */
  int K;           /* GLL nodes per element, 2..8 */
  double x0, x1;   /* physical domain, x0 < x1 */
  int bc;          /* DGFS_BC_PERIODIC or DGFS_BC_WALLS */
  double Tw[2];    /* side temperatures (left, right), > 0; DGFS_BC_WALLS only */
  double uw[6];    /* side velocities (left x, y, z, right x, y, z); 0 x components for walls */
  double acc[2];   /* wall accommodation coefficients in [0, 1]: 1 diffuse, 0 specular */
  int side[2];     /* DGFS_SIDE_WALL or DGFS_SIDE_INFLOW per side */
  const double* n_in; /* nullable [2 * s] in-flow densities (left side's s, then right's);
                         required for an in-flow side, >= 0 */
} dgfs_dg_desc;

/* Build a DG plan on top of a collision plan, which supplies the velocity grid (N, L),
 * the species and masses, the precision and the collision operator; the collision plan must
 * stay alive while the DG plan is used.  Allocates the step's work buffers on the collision
 * plan's device (2 * Ne * K * s * N^3 elements).  Errors: DGFS_ERR_INVALID_ARG (null or
 * out-of-range fields, s > 8), DGFS_ERR_OOM, DGFS_ERR_CUDA. */
int dgfs_dg_create(const dgfs_dg_desc* desc, dgfs_plan collision, dgfs_dg_plan* out);

/* Release a DG plan (waits for its work).  Null is accepted. */
int dgfs_dg_destroy(dgfs_dg_plan plan);

/* Physical positions of the Ne * K nodes (host array, element-major). */
int dgfs_dg_nodes(dgfs_dg_plan plan, double* x_out);

/* rhs = the transport part of d_t f (Eq. weakForm without its collision term): for every
 * element, node m and velocity, (2 / (h w_m)) [v_x sum_l S_ml f_l - flux terms of the faces].
 * f_dev and rhs_dev as described above; stream-ordered, asynchronous. */
int dgfs_dg_transport(dgfs_dg_plan plan, const void* f_dev, void* rhs_dev, void* stream);

/* One SSP-RK2 step of the full equation in place on f_dev:
 *   f1 = f + dt R(f),  f <- f/2 + (f1 + dt R(f1))/2,
 * R = transport + sum_j kappa_ij Q_ij, the collision term from the collision plan.  The
 * collision plan must have been created with DGFS_SUM_SPECIES (its kappa gives 1/Kn_ij) and
 * max_batch >= Ne * K, else DGFS_ERR_INVALID_ARG / DGFS_ERR_BUDGET.  Stream-ordered. */
int dgfs_dg_step(dgfs_dg_plan plan, void* f_dev, double dt, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DGFS_H */
