/*
 * bbdg.h -- C ABI of the GB300 (sm_103a) Bernstein-Bezier DG solver for the first-order
 * acoustic system (Chan & Warburton, "GPU-accelerated Bernstein-Bezier discontinuous
 * Galerkin methods for wave problems").
 *
 * The library evaluates, on one GPU, the per-stage right-hand side of the semi-discrete
 * system of Section 3 (eq. (discrete_var)) for the acoustic equations of Section 2,
 *
 *     p_t   = kappa [ -div u + sum_f (J^f/J^k) L^f F_p ]
 *     u_i,t = (1/rho) [ -d_i p + sum_f (J^f/J^k) n_i L^f F_u ],
 *     F_p = 1/2 (tau_p [p] - n.[u]),  F_u = 1/2 (tau_u [u].n - [p]),
 *     tau_p = 1/{rho c}, tau_u = {rho c},  mirror conditions p+ = -p-, u+ = u- on the
 *     domain boundary,
 *
 * with the Bernstein-Bezier derivative operators of Lemma 1 (4 nonzeros per row) and the
 * lift factored as L^f = E_L^f L0 and applied by one-degree reductions (Algorithm 1),
 * plus the low-storage RK4 update of Section 4.2, and a dense nodal (Warp & Blend)
 * right-hand side as the comparison path (Section 4.2, "node-per-thread" nodal kernels).
 *
 * Conventions shared by every call
 *   - State arrays are caller-owned DEVICE memory, contiguous, 16-byte aligned (any
 *     cudaMalloc / PyTorch allocation is), layout [S][K][N_p][4]: S shots, K elements,
 *     N_p = (N+1)(N+2)(N+3)/6 coefficients per field, and the four fields (p, u, v, w) of a
 *     coefficient adjacent (node-major, so one 16-byte access moves a node).
 *     The element type is double (BBDG_F64) or float (BBDG_F32), chosen at
 *     bbdg_setup_operators and applied to every state pointer.
 *   - S (shots) is in [0, 65535] and nsteps >= 0 (else BBDG_EINVAL); S = 0 or nsteps = 0
 *     is an empty batch: the call returns BBDG_OK at once, before any pointer check,
 *     and launches nothing.
 *   - Node order (BB basis): multi-index (a0,a1,a2,a3), |a| = N,
 *         for a0 in 0..N: for a1 in 0..N-a0: for a2 in 0..N-a0-a1: a3 = N-a0-a1-a2.
 *     The nodal basis uses the Warp & Blend node of the same multi-index.
 *   - Local vertex m of EToV <-> barycentric lambda_m <-> reference vertex
 *     v0=(-1,-1,-1), v1=(1,-1,-1), v2=(-1,1,-1), v3=(-1,-1,1); face m is the face
 *     opposite vertex m (lambda_m = 0).
 *   - Every call returns 0 (BBDG_OK) or a negative status; bbdg_last_error() gives the
 *     message.  No call aborts or exits.  Calls that take a stream only enqueue work on
 *     it (stream-ordered, no host synchronisation) unless stated otherwise.
 *   - A context is not thread-safe: use one context per host thread.
 */
#ifndef BBDG_H
#define BBDG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bbdg_ctx bbdg_ctx;

/* status codes */
#define BBDG_OK 0
#define BBDG_EINVAL (-1)       /* bad argument (null pointer, size, unsupported combination) */
#define BBDG_EUNSUPPORTED (-2) /* N outside [1, 10], unknown basis / precision / variant     */
#define BBDG_EMESH (-3)        /* non-positive Jacobian, non-manifold or unmatched face      */
#define BBDG_ECUDA (-4)        /* a CUDA runtime call failed (message has the CUDA error)    */
#define BBDG_ENOMEM (-5)       /* device or host allocation failed                           */
#define BBDG_ESTATE (-6)       /* call made before the setup it needs                        */
#define BBDG_ETIMEOUT (-7)     /* a bounded wait inside a kernel gave up (bbdg_device_status) */

/* bases, precisions, lift variants, flux */
#define BBDG_BB 0
#define BBDG_NODAL 1
#define BBDG_NODAL_TC 2   /* nodal basis, dense products on the tensor cores (FP32 only)      */
#define BBDG_F64 0
#define BBDG_F32 1
#define BBDG_F32_LIFT64 2     /* FP32 state and arithmetic, L0 and the reduction chain in FP64 */
#define BBDG_LIFT_OPTIMAL 0   /* L0 then N one-degree reductions (Algorithm 1)              */
#define BBDG_LIFT_SPARSE_EL 1 /* L0, then each node's row of the sparse lift-reduction      */
                              /* matrix E_L (<= N^f_p + 3 non-zeros; Algorithm 3), N <= 6  */
#define BBDG_FLUX_UPWIND 0    /* tau_p = 1/{rho c}, tau_u = {rho c} (Section 2)             */
#define BBDG_FLUX_CENTRAL 1   /* tau_p = tau_u = 0 (energy-conserving; Section 2 with tau=0) */
#define BBDG_BC_MIRROR 0
#define BBDG_BC_ABSORBING 1

/* stage kernel forms (bbdg_set_stage_form) */
#define BBDG_FORM_GROUP 0     /* groups of E elements per CTA iteration                      */
#define BBDG_FORM_WARP 1      /* one element per warp, warp-level synchronisation only       */
#define BBDG_FORM_PIPE 2      /* warp-specialised: reduction chains of one element group run */
                              /* beside the update of the previous group (N <= 8)           */
#define BBDG_FORM_ROWS 3      /* BBDG_NODAL_TC only: the MMA's rows are (field, element)     */
                              /* pairs of 32 elements, its columns the nodes (N <= 6)       */
#define BBDG_FORM_THREAD 4    /* one element per thread, all in registers (N <= 2)          */

/*
 * bbdg_setup_mesh -- create a context from an affine tetrahedral mesh (Section 3).
 *   out     : receives the new context (set to NULL on failure).
 *   Nv, vxyz: HOST array [Nv][3] of vertex coordinates (double).
 *   K, EToV : HOST array [K][4] of vertex ids (int32, 0-based); any orientation.
 *             Elements with negative orientation are rejected (BBDG_EMESH): list each
 *             tetrahedron with det[v1-v0, v2-v0, v3-v0] > 0.
 *   rho, kappa: HOST arrays [K] of density and bulk modulus, constant per element
 *             (Section 2); both must be > 0.
 * Faces are matched by their sorted global vertex triples; a face seen once is a domain
 * boundary face and gets the boundary condition of bbdg_set_boundary (the mirror conditions
 * of Section 2 by default).  The library copies every
 * input; the caller may free them on return.  Selects the current CUDA device.
 */
int bbdg_setup_mesh(bbdg_ctx** out, int64_t Nv, const double* vxyz, int64_t K,
                    const int32_t* EToV, const double* rho, const double* kappa);

/*
 * bbdg_setup_operators -- build and upload the reference operators for order N.
 *   N           : 1..10.
 *   basis       : BBDG_BB (Section 3.1, Lemma 1 and Algorithm 1) or BBDG_NODAL (Lagrange
 *                 basis on Warp & Blend nodes, dense D^r, D^s, D^t and lift, Section 3.1), or
 *                 BBDG_NODAL_TC: the same nodal operators on the tensor cores.  The Warp &
 *                 Blend nodes are invariant under permutations of the barycentric
 *                 coordinates, so D^s, D^t and L^1..L^3 are D^r and L^0 with rows and
 *                 columns permuted: only [D^r | L^0] is applied, to gathered per-element
 *                 columns, in TF32 with a three-pass high/low split (FP32 accuracy); needs
 *                 BBDG_F32 (else BBDG_EUNSUPPORTED) and ignores the launch shape's E.
 *   precision   : BBDG_F64 or BBDG_F32 (state type and arithmetic), or BBDG_F32_LIFT64:
 *                 FP32 state and arithmetic except L0 and the reduction chain (Algorithm 1),
 *                 which run in FP64 and round once to FP32 (BB basis, BBDG_LIFT_OPTIMAL only).
 *                 Every state pointer is FP32 for BBDG_F32 and BBDG_F32_LIFT64.
 *   lift_variant: BBDG_LIFT_OPTIMAL (Algorithm 1: L0, then the N one-degree reductions,
 *                 one thread per face vector) or BBDG_LIFT_SPARSE_EL (Algorithm 3, the
 *                 non-optimal surface kernel of Section 4.2: L0 row-parallel, then every
 *                 node gathers its row of E_L; BB basis and N <= 6, else
 *                 BBDG_EUNSUPPORTED).  Both give the same right-hand side up to rounding.
 *                 Ignored for the nodal bases.
 * Sets the measured default launch shape and stage form for (N, basis, precision) (see
 * bbdg_set_launch_shape, bbdg_set_stage_form).  May be called again to change N, basis or
 * precision; device tables are replaced.  Host-synchronous (uploads complete before return).
 */
int bbdg_setup_operators(bbdg_ctx* ctx, int N, int basis, int precision, int lift_variant);

/*
 * bbdg_set_materials -- replace kappa and rho (the bulk modulus and density of the acoustic
 * system, Section 2, constant per element) and everything derived from them (the upwind
 * weights tau_p = 1/{rho c}, tau_u = {rho c} per face, with rho c = sqrt(kappa rho)).
 *   kappa, rho: DEVICE arrays of the context's GPU, FP64, [S_or_1][K] (medium s of shot s),
 *               8-byte aligned; every entry finite and > 0 (else BBDG_EINVAL, nothing
 *               changes).  Caller-owned: the library copies them before it returns.
 *   S_or_1    : 1 = one medium for every shot; S > 1 = one medium per shot, after which every
 *               stage call (bbdg_rhs, bbdg_step, bbdg_step_graph, bbdg_step_noalloc,
 *               bbdg_rk_stage) must pass exactly S shots (else BBDG_EINVAL), and the adjoint
 *               calls answer BBDG_EUNSUPPORTED until one medium is set again.  At most 65535.
 * Host-synchronous: waits for all work on the device first (the caller's writes to kappa and
 * rho on any stream), then checks the values, copies them and rewrites the element records
 * on the device.  A graph captured by bbdg_step_graph is rebuilt at its next call.  With
 * operators set up, one copy of the element records is kept per medium (S_or_1 x K x 192
 * bytes in FP32, twice that in FP64).
 */
int bbdg_set_materials(bbdg_ctx* ctx, const void* kappa, const void* rho, int64_t S_or_1);

/* bbdg_set_flux -- BBDG_FLUX_UPWIND (default) or BBDG_FLUX_CENTRAL. Host-synchronous. */
int bbdg_set_flux(bbdg_ctx* ctx, int flux);

/*
 * bbdg_set_boundary -- exterior state on boundary faces (all bases):
 *   BBDG_BC_MIRROR (default): p+ = -p-, u+ = u- (the mirror conditions of Section 2);
 *   BBDG_BC_ABSORBING: p+ = 0, u+ = 0, a zero exterior state that the upwind flux turns into
 *   an outflow condition (the boundary faces then dissipate 1/2 int (tau_p p^2 + tau_u u_n^2)).
 * The adjoint entry points need BBDG_BC_MIRROR (else BBDG_EUNSUPPORTED).  Host-synchronous;
 * a graph captured by bbdg_step_graph is rebuilt at its next call.
 */
int bbdg_set_boundary(bbdg_ctx* ctx, int bc);

/*
 * bbdg_set_launch_shape -- launch shape of the stage kernels.
 *   E              : elements per group (one group per CTA iteration); 0 = built-in default
 *                    for (N, precision).  BB basis: 1 <= E <= 31 and the group's shared
 *                    memory must fit; nodal basis: a multiple of 4 in [4, 64].
 *   shots_per_tile : batched runs order the groups as [shot tile][element group][shot in
 *                    tile], so that CTAs running at the same time share an element group's
 *                    geometry and neighbour traces in L2 across shots; 0 or 1 = shot-major.
 *                    Used only when it divides S (else 1).
 * Chosen by the autotuner (paper_1512_06025_gb300.autotune); the paper tunes the elements
 * per block of each kernel (K_V, K_S, K_U, Section 4.2).  Requires bbdg_setup_operators.
 */
int bbdg_set_launch_shape(bbdg_ctx* ctx, int E, int shots_per_tile);

/*
 * bbdg_set_stage_form -- which BB stage kernel runs bbdg_rhs / bbdg_rk_stage / bbdg_step.
 *   form          : BBDG_FORM_GROUP: the group kernel, launch shape from
 *                   bbdg_set_launch_shape;
 *                   BBDG_FORM_WARP: each warp owns one element and runs the trace gather and
 *                   fluxes, L0 and the gradient coefficients, the reduction chain of
 *                   Algorithm 1 (one layer of the 8 face vectors at a time across the lanes)
 *                   and the update with __syncwarp only.  The paper's implementation section
 *                   tried element-per-thread Bernstein lift kernels and left more efficient
 *                   element-wise forms to future work; this is the element-per-warp one;
 *                   BBDG_FORM_PIPE: the warp-specialised group kernel: two warps per CTA run
 *                   L0 and the reduction chains of one element group while six warps
 *                   compute the gradient coefficients and the update of the group before it
 *                   and the fluxes of the group after it (shared-memory rings filled by bulk
 *                   copies, bounded mbarrier waits: see bbdg_device_status); N <= 8, a fixed
 *                   launch shape per (precision, N);
 *                   BBDG_FORM_ROWS (basis BBDG_NODAL_TC, N <= 6): the tensor-core nodal stage
 *                   with the MMA operands exchanged: its 128 rows are the 4 fields of 32
 *                   elements, its columns the nodes, and the full operator
 *                   [D^r D^s D^t L^0..L^3] (no symmetry permutations) the streamed operand;
 *                   for BBDG_NODAL_TC, BBDG_FORM_GROUP is the node-row kernel;
 *                   BBDG_FORM_THREAD (BB basis, N <= 2): one thread per (shot, element) runs
 *                   the whole stage in registers (compile-time indices), no shared memory,
 *                   no block barriers.
 *   warps_per_cta : 1..16, BBDG_FORM_WARP only (its shared memory, W (16 N_p + 4 N_p^{N-1}
 *                   + 8 (N^f_p|1) + 40) words of the state type plus tables, must fit).
 * All forms give the group kernel's results up to rounding (the sums are the same; the
 * compiler may contract them into fused multiply-adds in another order).
 * BBDG_FORM_WARP and BBDG_FORM_PIPE need the BB basis, BBDG_F64 or BBDG_F32 and
 * BBDG_LIFT_OPTIMAL (BBDG_FORM_THREAD also N <= 2), BBDG_FORM_ROWS the BBDG_NODAL_TC basis
 * with N <= 6 (else
 * BBDG_EUNSUPPORTED).  bbdg_setup_operators sets the measured
 * faster form: BBDG_FORM_WARP (4 warps per CTA) for the BB basis in BBDG_F64 with
 * BBDG_LIFT_OPTIMAL at N = 10, BBDG_FORM_THREAD for the BB basis in BBDG_F64 or
 * BBDG_F32 with BBDG_LIFT_OPTIMAL at N <= 2, BBDG_FORM_ROWS for BBDG_NODAL_TC at N <= 5,
 * BBDG_FORM_GROUP otherwise.
 * Host-synchronous; a graph captured by bbdg_step_graph is rebuilt at its next call.
 */
int bbdg_set_stage_form(bbdg_ctx* ctx, int form, int warps_per_cta);

/*
 * bbdg_set_sources -- point sources f = delta(x - x_s) r(t) added to the pressure
 * equation of shot shot[s] (not in the paper, which sets f = 0; Section 2):
 *   r(t) = (1 - 2 pi^2 f0^2 (t - t0)^2) exp(-pi^2 f0^2 (t - t0)^2)   (Ricker wavelet),
 * projected as kappa_e r(t) M^{-1} b / J^e onto the lowest-index element e that contains
 * x_s (all barycentric coordinates >= -1e-12), b_alpha = B_alpha(x_s).
 *   n   : number of sources (0 clears them).
 *   xyz : HOST [n][3] locations;  shot: HOST [n] shot index of each source (0 <= shot).
 * Requires bbdg_setup_operators (the projection depends on N).  Host-synchronous.
 */
int bbdg_set_sources(bbdg_ctx* ctx, int64_t n, const double* xyz, const int64_t* shot,
                     double f0, double t0);

/*
 * bbdg_set_receivers -- pressure receivers p(x_r) = sum_alpha q_alpha B_alpha(x_r),
 * evaluated in the lowest-index element containing x_r.  HOST [n][3].  Requires
 * bbdg_setup_operators and the BB basis.  Host-synchronous.
 */
int bbdg_set_receivers(bbdg_ctx* ctx, int64_t n, const double* xyz);

/*
 * bbdg_rhs -- rhs = A q + s(t): the semi-discrete right-hand side of eq. (discrete_var)
 * (plus the point sources evaluated at time t) for S shots.
 *   q, rhs : DEVICE [S][K][N_p][4] (precision of the context); must not alias.
 *   stream : cudaStream_t (NULL = legacy default stream).
 */
int bbdg_rhs(bbdg_ctx* ctx, const void* q, void* rhs, int64_t S, double t, void* stream);

/*
 * bbdg_step -- nsteps low-storage RK4 steps (Carpenter & Kennedy, five stages; Section 4.2):
 *   for s = 1..5: res = a_s res + dt (A q + s(t + c_s dt)); q = q + b_s res,
 * with t = t0 + n dt at step n.  Each stage is one fused kernel (trace gather, upwind
 * flux, volume derivatives, L0 and the reduction chain, update) that writes the new q to
 * the other buffer of the pair (q, scratch).
 *   q       : DEVICE [S][K][N_p][4], in: state at t0, out: state at t0 + nsteps dt.
 *   res     : DEVICE, same shape: the RK residual register.  a_1 = 0, so the first stage
 *             of every step overwrites it without reading it: its contents on entry are
 *             ignored (no need to zero it), and on return it holds the last stage's residual.
 *   scratch : DEVICE, same shape: ping-pong buffer (contents undefined on return).
 *   traces  : DEVICE [nsteps][S][nrec] receiver samples after each step (type of the
 *             context), or NULL.
 * For an odd nsteps the final state is copied back from scratch into q (one device-to-
 * device copy on the stream).  Works for both bases; point sources and receivers need the
 * BB basis.  q, res, scratch and traces must not alias.
 */
int bbdg_step(bbdg_ctx* ctx, void* q, void* res, void* scratch, int64_t S, double t0,
              double dt, int nsteps, void* traces, void* stream);

/*
 * bbdg_step_host -- bbdg_step on a state held in HOST memory: on the stream, copies q_host
 * into work, runs the nsteps steps there, and copies the final state back into q_host (and
 * the receiver traces into traces_host).  The call returns once everything is enqueued;
 * q_host holds the result after the stream has reached this point (synchronise the stream
 * or an event recorded after the call before reading it).
 *   q_host      : HOST [S][K][N_p][4] (precision of the context), in: state at t0, out:
 *                 state at t0 + nsteps dt.  Page-locked memory (cudaHostAlloc or
 *                 cudaHostRegister) lets the copies run asynchronously and overlap work on
 *                 other streams; pageable memory works, with the driver staging each copy.
 *   work        : DEVICE, caller-owned, 16-byte aligned, at least 3 state arrays
 *                 (3 S K N_p 4 sizeof(T) bytes: q, res, scratch), plus nsteps S nrec
 *                 sizeof(T) bytes for the traces when traces_host is given.  Contents on
 *                 entry are ignored (a_1 = 0: the residual register is never read first).
 *   traces_host : HOST [nsteps][S][nrec] receiver samples after each step, or NULL.
 * Independent batches on independent streams, each with its own work buffer and host
 * arrays, may be in flight at the same time (their copies and steps overlap).  Errors as
 * bbdg_step; BBDG_EINVAL also for a misaligned work pointer.
 */
int bbdg_step_host(bbdg_ctx* ctx, void* q_host, void* work, int64_t S, double t0, double dt,
                   int nsteps, void* traces_host, void* stream);

/*
 * bbdg_step_graph -- bbdg_step captured into a CUDA graph: the first call with a given set
 * of arguments (pointers, S, t0, dt, nsteps; launch shape, flux, boundary, stage form,
 * materials, sources, receivers and operators, whose setters drop the graph) records the whole sequence
 * of 5 x nsteps stage kernels (and receiver samples) into a graph owned by ctx; later calls
 * with the same arguments replay it with one graph launch on the stream.  Results are those
 * of bbdg_step.  The capture runs on a private stream of ctx; source amplitudes are baked
 * into the graph at capture time (t0, dt are part of the key).
 */
int bbdg_step_graph(bbdg_ctx* ctx, void* q, void* res, void* scratch, int64_t S, double t0,
                    double dt, int nsteps, void* traces, void* stream);

/*
 * bbdg_step_noalloc -- bbdg_step for callers that cannot allocate device memory: the
 * ping-pong buffer of the stages comes from a fixed array inside the library instead of
 * from the caller.  The paper has no counterpart; this exists for plug-ins that must not
 * use their host application's device allocator (the host owns all device memory) and for
 * real-time loops that forbid allocation after start-up (an allocation can block or fail
 * mid-run).
 *   q, res, S, t0, dt, nsteps, stream: as for bbdg_step (no scratch, no receivers).
 * Limit: S * K * 4 * N_p * sizeof(state type) must not exceed
 * bbdg_step_noalloc_max_bytes() (64 MiB); larger states are rejected with BBDG_EINVAL and a
 * message.  The array is a static device array of the library: every GPU that loads the
 * library holds it until the process exits.  Its address is looked up once per device, on
 * the first call made with that device current; make that first call before any stream
 * capture.  All calls share the array and it keeps the last call's contents (nothing in it
 * needs to start at zero): calls that overlap on the GPU (other streams or threads) race
 * on it and must be serialised by the caller.  Calls no cudaMalloc or cudaFree.
 */
int bbdg_step_noalloc(bbdg_ctx* ctx, void* q, void* res, int64_t S, double t0, double dt,
                      int nsteps, void* stream);

/* bbdg_step_noalloc_max_bytes -- size in bytes of the static array bbdg_step_noalloc uses. */
size_t bbdg_step_noalloc_max_bytes(void);

/*
 * bbdg_rk_stage -- one stage s (0..4) of the LSERK4 step of bbdg_step, as one fused kernel:
 *   res = a_s res + dt (A q_in + s(t + c_s dt));  q_out = q_in + b_s res.
 * t is the time at the start of the step.  q_in and q_out are two different DEVICE
 * buffers (neighbour traces of q_in are read while q_out is written); res is updated in
 * place (stage 0 has a_1 = 0 and only writes it: the kernels skip the read).  Five calls
 * with q_in/q_out swapped after each call make one step; this lets a caller build its own
 * loop or CUDA graph without the copy that bbdg_step needs for an odd number of steps.  Works for both bases (point sources need the BB basis).
 */
int bbdg_rk_stage(bbdg_ctx* ctx, const void* q_in, void* q_out, void* res, int64_t S, int stage,
                  double t, double dt, void* stream);

/*
 * bbdg_sample_receivers -- traces[s][r] = p(x_r) of shot s for state q (DEVICE).
 */
int bbdg_sample_receivers(bbdg_ctx* ctx, const void* q, void* traces, int64_t S, void* stream);

/*
 * bbdg_adjoint_rhs -- out = A^T mu: the transpose of the semi-discrete operator of
 * bbdg_rhs (without sources), for the discrete adjoint (reverse mode of eq.
 * (discrete_var); the paper is forward-only).  mu, out: DEVICE [S][K][N_p][4], FP64, must
 * not alias.  Needs the BB basis in FP64.  Uses library-owned work buffers (allocated on
 * first use, sized for S).
 */
int bbdg_adjoint_rhs(bbdg_ctx* ctx, const void* mu, void* out, int64_t S, void* stream);

/*
 * bbdg_adjoint_step -- reverse mode of one LSERK4 step of bbdg_step (five stages in
 * reverse order):  for s = 5..1:  mu = lam_res + b_s lam_q;  lam_res = a_s mu;
 * lam_q += dt A^T mu;  grad_kappa += dt (d(A q_{s-1} + f(t + c_s dt)) / d kappa)^T mu,
 * where A depends on kappa through the kappa scaling of the pressure equation, through
 * tau_p = 1/{rho c} and tau_u = {rho c} (c = sqrt(kappa / rho)) on both sides of every
 * face, and through the point sources.
 *   lam_q, lam_res : DEVICE [S][K][N_p][4] FP64 adjoint state, updated in place
 *                    (in: adjoints of the step's output, out: of its input).
 *   q_stages       : DEVICE [5][S][K][N_p][4] the forward inputs of the step's five stages
 *                    (q_{s-1}), or NULL when no gradient is wanted.
 *   grad_kappa     : DEVICE [K] FP64, accumulated (d J / d kappa_k), or NULL; needs S == 1.
 *   t, dt          : start time and step of the forward step.
 *   rec_residual   : DEVICE [nrec] FP64 or NULL: dJ/dp_r at the end of this step (for
 *                    J = 1/2 sum (p_r - d_r)^2: p_r - d_r), added as lam_q += R^T r first.
 * Needs the BB basis in FP64 and S == 1 when a gradient or residual is passed.
 */
int bbdg_adjoint_step(bbdg_ctx* ctx, void* lam_q, void* lam_res, const void* q_stages,
                      double* grad_kappa, int64_t S, double t, double dt,
                      const void* rec_residual, void* stream);

/*
 * bbdg_misfit -- the receiver misfit of the gradient form (not in the paper, which is
 * forward-only): resid[i] = traces[i] - data[i] and J = 1/2 sum_i resid[i]^2 for n values,
 * in FP64 with compensated (Neumaier) summation in a fixed order, so J is reproducible bit
 * for bit.  traces, data, resid: DEVICE double [n] (resid may alias traces); J: DEVICE
 * double [1], written.  One CTA, stream-ordered.  BBDG_EINVAL for NULL pointers or n < 0.
 */
int bbdg_misfit(bbdg_ctx* ctx, const void* traces, const void* data, int64_t n, void* resid, void* J,
                void* stream);

/* bbdg_last_error -- message of the last failing call on ctx (or of the last failing
 * bbdg_setup_mesh when ctx is NULL).  Valid until the next call on ctx. */
const char* bbdg_last_error(const bbdg_ctx* ctx);

/* bbdg_device_status -- BBDG_OK, or BBDG_ETIMEOUT once a bounded wait inside one of ctx's
 * kernels has given up since setup (the BBDG_NODAL_TC kernels then write NaN outputs for
 * the elements they could not finish; the BBDG_FORM_PIPE stage kernel goes on with the
 * stale contents of the shared-memory slot it waited for, so its outputs for that launch
 * are unreliable).  Only those two kernel families wait on the hardware (mbarrier waits on
 * bulk copies and tensor-core commits).  Synchronous: reads the status words from the
 * device after the work queued so far on the legacy default stream. */
int bbdg_device_status(bbdg_ctx* ctx);

/* bbdg_destroy -- free every device and host resource of ctx (NULL is a no-op). */
void bbdg_destroy(bbdg_ctx* ctx);

/*
 * bbdg_measure_fma_peak -- measured fused multiply-add rate of the current device, in
 * TFLOP/s (an FMA counts 2), for precision BBDG_F64 or BBDG_F32: the arithmetic roofline
 * denominator of kernels bound by the FP64 (or FP32) pipe (the paper's roofline study,
 * Section 4.4, divides by the peak of its GPU; here it is measured on the running one).
 * Runs a kernel of independent FMA chains on a grid of 8 CTAs per SM for about 60 ms after
 * a sizing launch; host-synchronous; allocates and frees a small device buffer.
 * BBDG_EINVAL for a NULL pointer or another precision, BBDG_ECUDA / BBDG_ENOMEM on
 * failures of the CUDA runtime.
 */
int bbdg_measure_fma_peak(int precision, double* tflops);

/* bbdg_num_nodes -- N_p for order N (0 if N is outside [1, 10]). */
int bbdg_num_nodes(int N);

/* bbdg_nodal_nodes -- barycentric coordinates [N_p][4] (HOST, double) of the Warp & Blend
 * nodes the nodal basis uses, in node order. */
int bbdg_nodal_nodes(int N, double* lam_out);

#ifdef __cplusplus
}
#endif
#endif /* BBDG_H */
