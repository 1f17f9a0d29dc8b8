/*
 * esdg.h -- C ABI of the GB300 entropy-stable DG (ESDG) shallow-water library.
 *
 * Method: Wu, Kubatko, Chan, "High-order entropy stable discontinuous Galerkin
 * methods for the shallow water equations: curved triangular meshes and GPU
 * acceleration" (arXiv 2005.02516).  The library evaluates the per-stage
 * right-hand side of the modal ESDG scheme, eq. (dgform) of Sec. 2.8, and
 * advances it with the low-storage RK45 scheme named in Sec. 4, on one GPU.
 *
 * Conventions shared by every call:
 *   - Every function returns an int status: ESDG_OK (0) or a negative code
 *     below.  No call throws or aborts; esdg_last_error() gives a message.
 *   - Host pointers are owned by the caller and are only read or written
 *     during the call.  Device pointers named as such are owned by the caller
 *     unless stated otherwise; library-owned device memory is released by
 *     esdg_destroy().
 *   - Arrays are dense, C order.  The state is u[field][element][mode], FP64,
 *     fields (h, hu, hv), modes of the orthonormal Dubiner basis in the order
 *     i = 0..N, j = 0..N-i (phi_ij = sqrt(2) P_i(a) P_j^(2i+1,0)(b) (1-b)^i,
 *     a = 2(1+r)/(1-s) - 1, b = s).  With ESDG_METHOD_SBP the last index runs
 *     over the Nq SBP nodes instead (state [3][K][Nq] of nodal values), and
 *     every [3][K][Np] state or right-hand side below is [3][K][Nq].
 *   - All work is enqueued on the stream given to esdg_attach_device(); calls
 *     that return host data synchronise that stream.
 */
#ifndef ESDG_H
#define ESDG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define ESDG_OK            0
#define ESDG_EINVAL       -1  /* bad argument, unsupported size, malformed mesh */
#define ESDG_ENOMEM       -2  /* host or device allocation failed / buffer too small */
#define ESDG_ECUDA        -3  /* a CUDA runtime call failed (message names it) */
#define ESDG_ENONPOSITIVE -4  /* the device found an entropy-projected depth <= 0 */
#define ESDG_ENONFINITE   -5  /* the device found a non-finite value */
#define ESDG_ESTATE       -6  /* call out of order (e.g. no device memory attached) */
#define ESDG_ETIMEOUT     -7  /* a bounded device-side wait (on an asynchronous copy) expired;
                                 the kernel stopped early and the state is not valid;
                                 copies into shared memory that the wait gave up on may
                                 still have been in flight when the block exited, so
                                 destroy the context (and, to be safe, the CUDA context)
                                 rather than reuse it; or a host-side wait
                                 (esdg_server_drain) ran out */
#define ESDG_EBUSY        -8  /* admission refused: the request's device footprint exceeds
                                 the server's whole HBM budget */

/* arithmetic of the right-hand side; state and RK accumulation are always FP64 */
#define ESDG_FP64 0
#define ESDG_FP32 1

/* built-in forcing terms */
#define ESDG_FORCING_NONE     0
#define ESDG_FORCING_MMS_SINE 1  /* manufactured solution h = 2 + a sin(pi(x+y-t)), u=u0, v=v0,
                                    b = bamp cos(pi x) cos(pi y): forcing added to du/dt */

/* volume quadrature rules (Sec. 2.1 asks for positive weights, exact to >= 2N-1) */
#define ESDG_RULE_COLLAPSED 0  /* collapsed Gauss rule, (N+1)^2 points, exact to degree 2N+1 */
#define ESDG_RULE_SYMMETRIC 1  /* fully symmetric interior rule exact to degree 2N:
                                  3, 6, 12, 16, 25 points for N = 1..5 */

/* domain boundary (Sec. 2.9): periodic, or reflective walls on all four
   sides (exterior state h+ = h, u_n+ = -u_n, tangential velocity kept) */
#define ESDG_BOUNDARY_PERIODIC 0
#define ESDG_BOUNDARY_WALLS 1

/* inverse curved mass matrix of the projection (Sec. 2.6) and the update
   (eq. (dgform)): the stored per-element inverse (M_h^k)^{-1} (Sec. 2.7), or
   the weight-adjusted inverse M^{-1} M_{1/J} M^{-1} = Vq^T W diag(1/J) Vq
   applied on the fly, the alternative Sec. 2.8 names (no per-element matrix
   is stored or read).  The weight-adjusted inverse keeps the entropy identity
   exact and conserves sum_k 1^T M~_k h_k (M~_k its inverse).  It equals the
   stored inverse on affine elements and for the symmetric rules of N = 1, 2
   (as many points as modes); a lake at rest stays exact where J is in P^N
   (affine elements, N <= 2) and elsewhere holds to the approximation error. */
#define ESDG_MASS_EXACT           0
#define ESDG_MASS_WEIGHT_ADJUSTED 1

/* the scheme: the hybridized modal ESDG method of Sec. 2 (unknowns: modal
   coefficients, state [3][K][Np]), or the traditional entropy-stable DG-SBP
   method of Sec. 3 (unknowns: nodal values at the Nq points of an SBP rule,
   exact to 2N-1 with the face Gauss-Legendre points among its nodes: 6, 10,
   18, 22, 34 points for N = 1..5; state [3][K][Nq]; no entropy projection;
   SBP operators Q_SBP = [I; I_f]^T Q_h [I; I_f] of Theorem 3.1; diagonal mass
   W J).  The DG-SBP method takes periodic boundaries and ESDG_MASS_EXACT,
   ignores volume_rule, and runs outside ensembles and the server.  Its
   ESDG_POINTS_VOLQ points are the SBP nodes, where initial data are given. */
#define ESDG_METHOD_MODAL 0
#define ESDG_METHOD_SBP   1

/* esdg_config.dense: how the FP32 modal path (stored inverse mass) applies
 * the shared dense operators Vq, Vq^T, Vh and the lift Vh^T (Sec. 2.6, 2.8).
 * ESDG_DENSE_TENSOR runs them on the tensor cores (tcgen05 MMA, TF32 operands
 * split into two parts, three products per step, FP32 accumulation in tensor
 * memory); it needs Np <= 16 and Nq <= 16 (N <= 4 with the symmetric rule,
 * N <= 3 with the collapsed one) and is refused elsewhere.  ESDG_DENSE_SIMT
 * runs them on the FP32 pipes.  ESDG_DENSE_AUTO (0) takes the faster of the
 * two, which on GB300 is the FP32 pipes at every degree where both exist.
 * FP64, DG-SBP and weight-adjusted contexts ignore the field.  Ensembles and
 * the request server apply the operators on the FP32 pipes whatever the
 * members ask. */
#define ESDG_DENSE_AUTO   0
#define ESDG_DENSE_SIMT   1
#define ESDG_DENSE_TENSOR 2

/* point sets for esdg_get_points */
#define ESDG_POINTS_NODAL 0  /* degree-N equispaced nodes, [K][Np] */
#define ESDG_POINTS_VOLQ  1  /* volume quadrature points,  [K][Nq] */
#define ESDG_POINTS_FACEQ 2  /* face quadrature points,    [K][Nfq] */

/* esdg_init_state modes */
#define ESDG_INIT_DEPTH   0  /* q[0] is the depth h */
#define ESDG_INIT_SURFACE 1  /* q[0] is the free surface H = h + b (exact lake at rest) */

typedef struct esdg_config {
    int N;                  /* polynomial degree, 1..5 */
    int precision;          /* ESDG_FP64 or ESDG_FP32 right-hand-side arithmetic */
    int nx, ny;             /* quads of the structured grid, each >= 3; K = 2 nx ny triangles */
    double x0, x1, y0, y1;  /* periodic domain [x0,x1] x [y0,y1] */
    double warp_ax, warp_ay;/* curving amplitudes (0 = affine mesh), see below */
    double g;               /* gravity */
    double cfl;             /* dt = cfl * ((x1-x0)/nx) / ((N+1)(N+2)/2), Sec. 4 */
    int lax_friedrichs;     /* 1: add the local Lax-Friedrichs penalty (entropy stable),
                               0: entropy-conservative flux alone */
    int forcing;            /* ESDG_FORCING_* */
    double mms_amp, mms_bamp, mms_u0, mms_v0;  /* ESDG_FORCING_MMS_SINE parameters */
    int volume_rule;        /* ESDG_RULE_* */
    int boundary;           /* ESDG_BOUNDARY_* */
    int mass;               /* ESDG_MASS_*; ensembles and served FP32 requests take ESDG_MASS_EXACT */
    int method;             /* ESDG_METHOD_* */
    int dense;              /* ESDG_DENSE_* (FP32 modal path with the stored inverse) */
} esdg_config;

/*
 * Mesh: quad (i,j), q = j*nx + i, splits along its lower-left to upper-right
 * diagonal into elements 2q = (v(i,j), v(i+1,j), v(i+1,j+1)) and
 * 2q+1 = (v(i,j), v(i+1,j+1), v(i,j+1)), mapped from the reference vertices
 * (-1,-1), (1,-1), (-1,1).  Curved elements: the degree-N equispaced nodes of
 * each affine element are moved by, with xi = 2(x-xc)/Lx, eta = 2(y-yc)/Ly,
 *     x += warp_ax * Lx/2 * cos(pi xi / 2) cos(3 pi eta / 2)
 *     y += warp_ay * Ly/2 * sin(2 pi xi)   cos(pi eta / 2)
 * and the element map is their degree-N interpolant (Sec. 2.7, Sec. 4).
 */

typedef struct esdg_ctx esdg_ctx;

/*
 * esdg_build_operators -- build on the host, in FP64, the reference-element
 * operators of Sec. 2.1-2.3 (V_q, V_f, P_q, Q-hat, hybridized Q_h), the mesh,
 * the geometric factors and (M_h^k)^{-1} of Sec. 2.7.  Validates J > 0 at every
 * quadrature node and that every face node has a matching neighbour node
 * (ESDG_EINVAL otherwise).  *out receives a new context; no device work.
 */
int esdg_build_operators(const esdg_config* cfg, esdg_ctx** out);

/* The configuration the context was built with. */
int esdg_get_config(const esdg_ctx* ctx, esdg_config* out);

/* Sizes: K elements, Np modes, Nq volume and Nfq face quadrature points, and
 * the device bytes that esdg_attach_device() needs.  Any pointer may be NULL. */
int esdg_sizes(const esdg_ctx* ctx, int* K, int* Np, int* Nq, int* Nfq, size_t* device_bytes);

/*
 * esdg_attach_device -- give the library its device memory and stream, and
 * upload operators and geometry.  device_buffer: caller-owned device memory of
 * at least esdg_sizes(...device_bytes) bytes, 256-byte aligned, kept alive
 * until esdg_destroy(); or NULL, in which case the library allocates (and later
 * frees) that memory itself.  stream: a cudaStream_t (NULL = legacy default).
 */
int esdg_attach_device(esdg_ctx* ctx, void* device_buffer, size_t bytes, void* stream);

/* Physical coordinates of a point set (ESDG_POINTS_*), host arrays [K][n]. */
int esdg_get_points(const esdg_ctx* ctx, int kind, double* x, double* y);

/*
 * esdg_init_state -- set bathymetry and initial state from host arrays.
 * b_nodal [K][Np]: bathymetry at the ESDG_POINTS_NODAL points; b is the degree-N
 * polynomial through these values on each element (C0 across elements when
 * shared nodes carry equal values, Sec. 4.1).  q_volq [3][K][Nq]: (h or H, hu,
 * hv) at the volume quadrature points, L2-projected with the J-weighted mass
 * matrix (Sec. 2.7).  mode ESDG_INIT_SURFACE sets h = Pi(H) - b so a lake at rest
 * is exact.  Resets the RK residual.
 */
int esdg_init_state(esdg_ctx* ctx, const double* b_nodal, const double* q_volq, int mode);

/* esdg_prepare -- the host work of esdg_init_state done before any device
 * memory exists: builds, in host memory, the complete image of operators,
 * geometry, bathymetry and projected initial state, so that the next
 * esdg_attach_device is one host-to-device copy.  Arguments as for
 * esdg_init_state.  Call between esdg_build_operators and esdg_attach_device. */
int esdg_prepare(esdg_ctx* ctx, const double* b_nodal, const double* q_volq, int mode);

/* Bathymetry alone (b_nodal as above); keeps the state. */
int esdg_set_bathymetry(esdg_ctx* ctx, const double* b_nodal);

/* Overwrite the modal state u [3][K][Np] FP64 from host (on_device = 0) or
 * device (on_device = 1) memory; resets the RK residual. */
int esdg_set_state(esdg_ctx* ctx, const double* u, int on_device);

/* Copy the modal state out, to host (on_device = 0) or device memory. */
int esdg_copy_state(const esdg_ctx* ctx, double* u, int on_device);

/*
 * esdg_rhs -- one evaluation of the semi-discrete right-hand side du/dt of
 * eq. (dgform) (Sec. 2.8) at time t: entropy projection (Sec. 2.6), flux
 * differencing with the entropy-conservative SWE flux and its well-balanced
 * bathymetry term, interface flux plus Lax-Friedrichs, lift and inverse curved
 * mass matrix, plus the forcing if configured.  u_in: device [3][K][Np] FP64 or
 * NULL for the current state.  rhs_out: device [3][K][Np] FP64.  Synchronises
 * the stream and returns ESDG_ENONPOSITIVE / ESDG_ENONFINITE if the device
 * flagged a bad entropy-projected state.
 */
int esdg_rhs(esdg_ctx* ctx, double t, const double* u_in, double* rhs_out);

/*
 * esdg_step -- advance the current state by nsteps LSRK45 steps (five stages
 * each, Carpenter-Kennedy 2N-storage, Sec. 4) of size dt (dt <= 0: the CFL
 * rule of Sec. 4).  *t_inout is advanced.  The residual persists between
 * calls.  Synchronises the stream once at the end and reports device flags.
 */
int esdg_step(esdg_ctx* ctx, int nsteps, double dt, double* t_inout);

/*
 * esdg_step_host -- esdg_set_state + esdg_step + esdg_copy_state for a state
 * that lives in host memory, without separate copies: the projection kernel
 * reads u_host ([3][K][Np] FP64) directly over the host link and stores it as
 * the RK state (residual zeroed), nsteps steps run as in esdg_step, and the
 * last stage kernel writes the new state to u_out_host.  Both buffers must be
 * host memory the device can address (cudaHostAlloc / cudaHostRegister, or
 * managed memory), else ESDG_EINVAL; they may be the same buffer.
 * Synchronises once and reports device flags like esdg_step.
 */
int esdg_step_host(esdg_ctx* ctx, const double* u_host, int nsteps, double dt, double* t_inout, double* u_out_host);

/* Enqueue nsteps steps without synchronising or checking flags (for timing
 * loops and graph capture); esdg_check() reads the flags later. */
int esdg_step_async(esdg_ctx* ctx, int nsteps, double dt, double t0);
int esdg_check(esdg_ctx* ctx);

/*
 * esdg_entropy -- FP64 diagnostics of the current state (Sec. 2.4):
 * entropy = sum_k sum_q w_q J_q S(u_q), mass = sum_k sum_q w_q J_q h_q, and, if
 * entropy_rate is not NULL, the semi-discrete entropy rate
 * sum_k sum_q w_q J_q v(u_q) . (V_q du/dt)_q at time t (zero for the
 * entropy-conservative flux on a periodic mesh, Theorem 2.2).
 */
int esdg_entropy(esdg_ctx* ctx, double t, double* entropy, double* mass, double* entropy_rate);

/*
 * esdg_l2_error -- FP64 L2 error of the current state against values given at
 * the volume quadrature points (the error measure of the convergence study,
 * Sec. 4.1, evaluated with the element's own volume rule):
 *     err[f] = sqrt( sum_k sum_q w_q J_q^k (u_q[f] - exact_volq[f][k][q])^2 ),
 * f = 0, 1, 2 for (h, hu, hv); u_q = V_q u_h (modal) or the nodal values
 * (ESDG_METHOD_SBP, whose volume points are its nodes).
 * exact_volq: device memory [3][K][Nq] FP64 (values at the ESDG_POINTS_VOLQ
 * points, e.g. an exact solution), owned by the caller; host memory is refused
 * with ESDG_EINVAL.  err: host array of 3 doubles.  Uses the context's
 * diagnostic scratch; synchronises the stream.
 */
int esdg_l2_error(esdg_ctx* ctx, const double* exact_volq, double* err);

/*
 * Element partition of one solve (one GPU per block; the multi-GPU form of a
 * single solve: the elements of the structured grid split into px x py blocks
 * of whole quads, with one exchange of the entropy-projected face values per
 * RK stage, since the interface flux of Sec. 2.8 at a cut face needs the
 * neighbour's u~ on that face).
 *
 * esdg_build_partition -- the context of block `part` (0 <= part < px * py,
 * block (part % px, part / px); block b covers quads [b n / p, (b + 1) n / p) in
 * each direction) of the mesh cfg describes.  Its K local elements are the
 * block's, in increasing global order (global element 2 q + t of quad q =
 * j nx + i, as esdg_build_operators numbers them); its ghosts are the elements of
 * other blocks across a cut face, sorted by owning block, then global element.
 * All per-element calls (points, bathymetry, state, entropy, L2 error) act on
 * the local elements.  px = py = 1 is the whole mesh.  ESDG_EINVAL for a bad
 * block layout or configuration; no device work.  The block is cut out of the
 * whole mesh built on the host, so each caller pays the host set-up of the
 * whole mesh once (seconds at K = 131072) and keeps only its block.
 */
int esdg_build_partition(const esdg_config* cfg, int px, int py, int part, esdg_ctx** out);

/* K_global: elements of the whole mesh; nghost: ghost records; px, py, part
 * as built; trace_bytes: bytes of one face trace (the N+1 node records of one
 * face, 4 values each: the unit of the halo exchange).  Any output may be
 * NULL. */
int esdg_partition_info(const esdg_ctx* ctx, int* K_global, int* nghost, int* px, int* py, int* part,
                        size_t* trace_bytes);

/* Host arrays (any may be NULL): owned_gid [K] the global element of each local
 * element, ghost_gid [nghost] the global element of each ghost record,
 * ghost_part [nghost] the block that owns it. */
int esdg_partition_maps(const esdg_ctx* ctx, int* owned_gid, int* ghost_gid, int* ghost_part);

/* The face-neighbour table, host array [K][3]: 4 * element + face of the
 * neighbour across each face (4 * own element + 3 on a wall).  In a partition,
 * element indices >= K' = K rounded up to a multiple of 8 name ghost record
 * index - K'. */
int esdg_get_neighbors(const esdg_ctx* ctx, int* nbr);

/*
 * Per-stage stepping with a halo exchange in between (partitions; it works on
 * any context).  esdg_project: the entropy-projected values u~ of the current
 * state (Sec. 2.6) into the current u~ buffer.  esdg_stage: LSRK45 stage
 * `stage` (0..4, Sec. 4) of the step that starts at t0 with step dt: reads the
 * current u~ buffer (own and ghost records), updates u and the residual, and
 * writes the next stage's u~ into the other buffer, which becomes current.
 * ESDG_ESTATE before esdg_project.  A partition with ghosts must exchange its
 * halo after esdg_project and after every esdg_stage; esdg_step, esdg_rhs and
 * esdg_step_host refuse it (ESDG_ESTATE).  Asynchronous on the context's
 * stream; errors found on the device surface at esdg_check.
 */
int esdg_project(esdg_ctx* ctx);
int esdg_stage(esdg_ctx* ctx, int stage, double dt, double t0);

/* Halo exchange on the current u~ buffer, in face traces of trace_bytes (the
 * entropy-projected values at the N+1 nodes of one face: what the interface
 * flux of the element across that face reads).  esdg_halo_pack gathers the
 * traces of the n faces faces_dev[i] = 4 e + f (device int array; local
 * element e < K, face f < 3; an entry out of range gives zeros) into out_dev
 * (device, n traces); esdg_halo_unpack writes n traces from in_dev (device)
 * into the faces faces_dev[i] = 4 g + f of ghost records g < nghost (an entry
 * out of range is skipped).  Both asynchronous on the context's stream; the
 * caller owns the buffers. */
int esdg_halo_pack(esdg_ctx* ctx, const int* faces_dev, int n, void* out_dev);
int esdg_halo_unpack(esdg_ctx* ctx, const void* in_dev, const int* faces_dev, int n);

/*
 * esdg_entropy_noalloc -- the entropy and mass of esdg_entropy (no rate), for
 * callers that cannot allocate device memory while they run: code inside a
 * memory-pool or arena regime that forbids new allocations, or a driver loop
 * that must not call cudaMalloc/cudaFree between launches.  The paper has no
 * counterpart; this is a library convenience.
 *
 * u_dev: device state [3][K][Np] FP64, or NULL for the context's state; a
 * pointer that is not device (or managed) memory is refused with ESDG_EINVAL
 * before any launch.
 * entropy, mass: host outputs (either may be NULL).
 * Scratch: the per-block partial sums live in one file-scope device array of
 * ESDG_NOALLOC_MAX_PARTS * 3 + 4 doubles (about 96 KB), held by every GPU that
 * loads the library until the process exits.  One partial covers
 * ESDG_NOALLOC_POINTS_PER_PART volume quadrature points, so K * Nq must not
 * exceed ESDG_NOALLOC_MAX_PARTS * ESDG_NOALLOC_POINTS_PER_PART (ESDG_EINVAL
 * otherwise, checked on the host before the context's state and before any
 * CUDA call).  The call allocates nothing: no cudaMalloc, no cudaFree.
 * Every call looks up the array's device address with the caller's device
 * current (cudaGetSymbolAddress, which allocates nothing), so the address
 * stays valid across a device reset; the first call on a device may load the
 * library's device code, so make it before any stream capture.  Every call
 * overwrites the whole scratch it reads, but all calls
 * share the one array: calls that overlap on the GPU (other streams, other
 * threads) race and must be serialised by the caller.  Synchronises the
 * context's stream.
 */
#define ESDG_NOALLOC_MAX_PARTS 4096
#define ESDG_NOALLOC_POINTS_PER_PART 2048
int esdg_entropy_noalloc(const esdg_ctx* ctx, const double* u_dev, double* entropy, double* mass);

/*
 * Ensembles: several independent problems (contexts) of mixed degree N and
 * size K advanced together, one persistent kernel launch per RK stage over a
 * tile table of all members' element batches, the steps replayed from a
 * captured CUDA graph.  Members must be FP32 contexts, attached on the same
 * stream, with no forcing, all with the same volume rule.  Each member steps with its own CFL time step
 * (Sec. 4); members stay ordinary contexts (esdg_copy_state, esdg_entropy ...).
 * The ensemble allocates one small device table (a few hundred bytes per
 * member) with cudaMalloc and frees it in esdg_ensemble_destroy.
 */
typedef struct esdg_ensemble esdg_ensemble;
int esdg_ensemble_create(esdg_ctx* const* members, int n, esdg_ensemble** out);

/* Choose the launch shape (warps per CTA) and the order of members in the
 * tile table by timing candidate shapes on the members' current states (the
 * states are restored afterwards).  *warps and *order (0: as given,
 * 1: largest degree first) receive the choice; either may be NULL. */
int esdg_ensemble_autotune(esdg_ensemble* ens, int* warps, int* order);

/* Advance every member by nsteps LSRK45 steps; synchronises and checks the
 * members' device flags. */
int esdg_ensemble_step(esdg_ensemble* ens, int nsteps);
int esdg_ensemble_step_async(esdg_ensemble* ens, int nsteps);
int esdg_ensemble_destroy(esdg_ensemble* ens);

/* Message for the last failing call on ens (NULL: the last failing create). */
const char* esdg_ensemble_error(const esdg_ensemble* ens);

/*
 * Served form: a continuous-batching request loop on a worker thread.
 * A request is a context built with esdg_build_operators (not attached) plus
 * its host initial data (as for esdg_init_state) and a step count.  Requests
 * wait in a FIFO queue and are admitted when their device footprint
 * (esdg_sizes) fits the budget next to the active ones; device memory comes
 * from the stream-ordered allocator (cudaMallocAsync/cudaFreeAsync).  Each
 * iteration advances every active request by up to 20 steps (never past its
 * own step count): FP32 requests with 20 or more steps left together in one
 * ensemble launch per RK stage (per volume rule), an FP32 request with fewer
 * left through its own stage kernels, FP64 requests through their own stage
 * kernels on a stream of their own (created at admission), so that their
 * kernels overlap on the device.  Admission is FIFO and also stops while the
 * active requests of the head request's precision hold 2^23 (FP32) or 2^21
 * (FP64) unknowns per field (K Np) or more, so an overloaded server finishes
 * requests in arrival order rather than advancing all of them slowly (a
 * request is always admitted when none of its precision is active).  A
 * partition block (esdg_build_partition with ghosts) is refused with
 * ESDG_EINVAL.  A
 * finished request's state is copied to result_host ([3][K][Np] FP64) and its
 * device memory returned before queued requests are admitted.
 * Ownership of ctx passes to the server on a successful submit (it is
 * destroyed when the request finishes); b_nodal and q_volq are copied;
 * result_host must stay valid until the request is done.  FP32 requests
 * run in an ensemble and must be modal with the stored inverse and no forcing
 * term (else ESDG_EINVAL); FP64 requests take any configuration (each carries
 * its own simulated time for forcing terms); requests larger than the whole
 * budget are refused (ESDG_EBUSY).  Times are seconds since esdg_server_create.
 */
typedef struct esdg_server esdg_server;
int esdg_server_create(size_t hbm_budget_bytes, int max_active, void* stream, esdg_server** out);
int esdg_server_submit(esdg_server* srv, esdg_ctx* ctx, const double* b_nodal, const double* q_volq, int mode,
                       int nsteps, double* result_host, int* ticket);
/* state: 0 queued, 1 running, 2 done, < 0 failed with that status code. */
int esdg_server_query(esdg_server* srv, int ticket, int* state, double* t_submit, double* t_admit, double* t_done);
/* Wait until no request is queued or running (ESDG_ETIMEOUT after timeout_s). */
int esdg_server_drain(esdg_server* srv, double timeout_s);
/* iterations of the loop; steps: the sum over iterations of the most steps any
 * request advanced in it; bytes_in_use: device memory held by running requests;
 * max_active_seen: the most requests one iteration advanced together.  Any
 * output may be NULL. */
int esdg_server_stats(esdg_server* srv, long long* iterations, long long* steps, size_t* bytes_in_use,
                      int* max_active_seen);
/* Where the worker thread's time went, seconds since creation, into
 * seconds[0..4]: admission (device allocation and the copy of each prepared
 * image), ensemble rebuilds (membership changes), enqueueing each iteration's
 * work, waiting for the GPU, retiring results (status checks, result copies). */
int esdg_server_timing(esdg_server* srv, double* seconds);
/* Drops queued requests (state ESDG_ESTATE), ends running ones after their
 * current iteration (at most 20 steps; state ESDG_ESTATE, no result written),
 * releases everything. */
int esdg_server_destroy(esdg_server* srv);

/*
 * Volume-kernel cost comparison (Sec. 5.4): the traditional DG volume term
 * against the ESDG flux-differencing term with dense n x n operators (the
 * paper uses random entries), per element with n nodes:
 *   ESDG_VOLUME_DG:   out = Q^x f^x(u) + Q^y f^y(u)            (eq. (SWE) fluxes)
 *   ESDG_VOLUME_ESDG: out = (Q^x o F^x) 1 + (Q^y o F^y) 1,
 *                     F^i[j][k] = f_S^i(u_j, u_k)              (eqs. (SWE_flux1/2))
 * Qx, Qy: row-major [n][n] (Q[j][k] couples node k into row j); u, out:
 * [3][K][n] conservative (h, hu, hv) and result; element type float
 * (ESDG_FP32) or double (ESDG_FP64); h must be non-zero.  1 <= n <= 256.
 * esdg_volume_kernel takes device pointers and launches on `stream`
 * (asynchronous; ESDG_ECUDA on a launch failure); esdg_volume_kernel_host
 * takes host pointers and computes on the calling thread.  ESDG_EINVAL for a
 * bad kind, precision, size or null pointer.  Not part of the solver path.
 */
#define ESDG_VOLUME_DG 0
#define ESDG_VOLUME_ESDG 1
int esdg_volume_kernel(int kind, int precision, int n, int K, double g, const void* Qx, const void* Qy,
                       const void* u, void* out, void* stream);
int esdg_volume_kernel_host(int kind, int precision, int n, int K, double g, const void* Qx, const void* Qy,
                            const void* u, void* out);

/* The CFL time step of Sec. 4 for this configuration. */
int esdg_dt(const esdg_ctx* ctx, double* dt);

/* Release the context and any library-owned device memory. */
int esdg_destroy(esdg_ctx* ctx);

/* Message for the last failing call on ctx (ctx may be NULL for
 * esdg_build_operators failures).  The string lives until the next call. */
const char* esdg_last_error(const esdg_ctx* ctx);

/*
 * esdg_selftest_wait_timeout -- failure-detection self-test: one warp waits,
 * through the same bounded mbarrier wait that the stage kernels put on their
 * bulk copies, on a phase that no copy completes.  After its cycle limit
 * (about a second) the wait sets the timeout bit of a status word and the
 * kernel returns, with nothing in flight.  Returns ESDG_ETIMEOUT when that
 * happened (the expected outcome), ESDG_OK if the phase completed (it cannot),
 * ESDG_ECUDA / ESDG_ENOMEM on a CUDA failure.  stream: a cudaStream_t.
 */
int esdg_selftest_wait_timeout(void* stream);

#ifdef __cplusplus
}
#endif

#endif /* ESDG_H */
