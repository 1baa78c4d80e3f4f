/*
 * bgk.h -- C-ABI of libbgk: one explicit Runge--Kutta stage of the
 * six-dimensional Boltzmann--(ES-)BGK residual on hexahedral elements,
 * GB300 (sm_103a) native.
 *
 * Method: Dzanic & Martinelli, "Direct molecular gas dynamics simulations of
 * re-entry vehicles via the Boltzmann equation" (arXiv 2312.06567),
 * section "Methodology": flux-reconstruction (FR) advection u.grad f per
 * discrete velocity with the upwind interface flux and the DG-recovering
 * correction function, fused with the conservative BGK source (moments
 * Q = (rho, rho U, E), the modified state Q' of the discrete compatibility
 * condition, the ES-BGK equilibrium with the reduced F/G distributions).
 *
 * Conventions (every call):
 *  - Layouts.  Element e = e1 + n1 (e2 + n2 e3) of a uniform box mesh.
 *    Solution node s = i1 + (p+1)(i2 + (p+1) i3) at tensor Gauss--Legendre
 *    points.  Velocity node k = k1 + n1 (k2 + n2 k3) of a uniform grid.
 *    Point index P = e * Ns + s.  State f[c][k][e][s] (c = 0: F, c = 1: G,
 *    present only when delta > 0), contiguous, s fastest.
 *  - Precision.  BGK_FP64: state arrays are double.  BGK_MIXED: state arrays
 *    are float (the moment reduction and the Q' solve stay FP64-accurate).
 *    Moment / macroscopic arrays are always double.
 *  - Ownership.  The context owns every buffer it allocates.  Caller
 *    pointers are borrowed for the duration of the call, never retained.
 *  - on_device = 1: the pointer is device memory of the context's device
 *    (e.g. a torch tensor's data_ptr()); 0: host memory.
 *  - Streams.  All work is ordered on the stream given to bgk_create.  Calls
 *    that return host data synchronise that stream.
 *  - Errors are returned as bgk_status codes, never by trap or abort; the
 *    text of the last error is available from bgk_last_error.  A device-side
 *    failure (Newton non-convergence, non-finite state) is recorded in a
 *    device status word and reported by the next call that synchronises.
 */
#ifndef BGK_H
#define BGK_H

#if defined(__GNUC__)
#define BGK_API __attribute__((visibility("default")))
#else
#define BGK_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bgk_ctx bgk_ctx;

typedef enum {
    BGK_OK = 0,
    BGK_EINVAL = 1,    /* invalid argument or descriptor                       */
    BGK_ENOMEM = 2,    /* device allocation failed                             */
    BGK_ECUDA = 3,     /* a CUDA runtime call failed                           */
    BGK_ENOCONV = 4,   /* the Q' Newton iteration did not converge somewhere   */
    BGK_ETIMEOUT = 5,  /* a bounded wait inside a kernel gave up               */
    BGK_ENOTSUP = 6    /* valid but unsupported configuration                  */
} bgk_status;

typedef enum { BGK_FP64 = 0, BGK_MIXED = 1 } bgk_precision;

/* Hexahedral mesh of structured topology and FR order (section "Numerical
 * method": N_e elements, N_s = (p+1)^3 solution nodes each).  Element
 * e = e1 + n1 (e2 + n2 e3) has the face neighbours e +- 1, e +- n1,
 * e +- n1 n2 (wrapping on periodic axes).  Axes with periodic[d]=0 are
 * closed at both ends by weak faces (section "Implementation & problem
 * setup": exterior states enforced through the Riemann flux), chosen per
 * face 2d + (side > 0) by face_type:
 *   BGK_FACE_DIRICHLET: the exterior state is the Maxwellian of
 *     bc_state = (rho, U1, U2, U3, theta), G's delta theta / 2 times it;
 *   BGK_FACE_SPECULAR: a symmetry plane; the exterior state at velocity u
 *     is the element's own trace at u with its d-component negated (the
 *     velocity grid must be symmetric in axis d; uniform box only);
 *   BGK_FACE_DIFFUSE: a diffuse wall at bc_state = (unused, U_w1..3,
 *     theta_w): at each flux node the particles entering the gas come from
 *     rho_w M(u; U_w, theta_w) (G: delta theta_w / 2 times it), rho_w set so
 *     that no mass crosses the node (a reading: the paper names the
 *     condition only);
 *   BGK_FACE_CLOSED: a collapsed face of zero area (the pole of a
 *     latitude--longitude grid); no flux crosses it.
 * Geometry: node_xyz = NULL gives the uniform box lo..hi (hi[d] > lo[d]);
 * otherwise node_xyz[P][3] (host memory, P = N_e N_s, node s = i1 + (p+1)
 * (i2 + (p+1) i3) at the Gauss--Legendre points) are the coordinates of the
 * solution nodes, and each element's geometry is their interpolant of
 * degree p.  The library then forms the metric terms S^d = J grad xi_d in
 * the conservative curl form on the element's Gauss--Lobatto points and
 * runs FR on the equation mapped to the reference cube (transformed flux
 * (u . S^d) f, face vectors = the traces of S^d averaged over both sides):
 * conservative, and free-stream preserving when the geometry is continuous
 * across faces.  Diffuse and closed faces use the same (curvilinear) path
 * on the uniform box.  Specular faces are not available on it (BGK_ENOTSUP).
 * Requirements: n[d] >= 1, 1 <= order <= 4, J > 0 at every node. */
typedef struct {
    int n[3];
    double lo[3], hi[3];
    int periodic[3];
    int order;
    double bc_state[6][5];
    int face_type[6];           /* BGK_FACE_* per non-periodic face 2d + (side > 0) */
    const double *node_xyz;     /* NULL, or [P][3] solution-node coordinates (borrowed) */
} bgk_mesh_desc;

#define BGK_FACE_DIRICHLET 0
#define BGK_FACE_SPECULAR 1
#define BGK_FACE_DIFFUSE 2
#define BGK_FACE_CLOSED 3

/* Uniform Cartesian velocity grid with trapezoid weights (section
 * "Numerical method": discrete integration operator with strictly positive
 * entries, the trapezoidal rule on a uniform grid).  n[d] >= 2, hi > lo. */
typedef struct {
    int n[3];
    double lo[3], hi[3];
} bgk_vgrid_desc;

/* Gas (section "Governing equations"): delta internal degrees of freedom
 * (>= 0; delta > 0 carries the reduced pair F, G), Prandtl number Pr of the
 * ES-BGK temperature tensor (Pr >= 2/3 keeps it positive definite), and the
 * Sutherland law mu = mu_ref (theta/theta_ref)^(3/2) (theta_ref + theta_S) /
 * (theta + theta_S); theta_S < 0 selects mu = mu_ref.  tau = mu / (Pr P). */
typedef struct {
    double delta, Pr, mu_ref, theta_ref, theta_S;
} bgk_gas_desc;

/* Create a solver context on the current CUDA device for the problem as the
 * paper states it (section "Methodology": the mesh and FR order, the discrete
 * velocity set and its weights, the gas), with the state precision
 * BGK_FP64 or BGK_MIXED.  stream: a cudaStream_t (NULL = legacy default
 * stream).  Allocates three state copies (f^n and two stage buffers) plus
 * per-point work arrays; the descriptors are read during the call only.  On
 * failure *out may still hold a context whose bgk_last_error explains the
 * error; pass it to bgk_destroy.
 * Errors: BGK_EINVAL (descriptor), BGK_ENOMEM, BGK_ECUDA. */
BGK_API bgk_status bgk_create(bgk_ctx **out, const bgk_mesh_desc *mesh, const bgk_vgrid_desc *vgrid,
                      const bgk_gas_desc *gas, int precision, void *stream);
/* Synchronise the context's stream, release every device buffer, graph,
 * stream and event it owns, and free it.  Errors: BGK_EINVAL (NULL). */
BGK_API bgk_status bgk_destroy(bgk_ctx *ctx);

/* The metric terms the library builds for a curvilinear mesh (section
 * "Numerical method": FR on curved elements through the transformed flux;
 * host only, no context, no CUDA call): for mesh->node_xyz (required) and the FR order,
 * S[P][9] = (S^1, S^2, S^3) at each solution node (S^d = J grad xi_d, the
 * conservative curl form on the element's Gauss--Lobatto points evaluated at
 * the Gauss nodes), J[P] = det(dX/dxi) at the nodes, and the face vectors
 * fvec[N_e][6][(p+1)^2][3] (face 2d + (side > 0), oriented along +xi_d, the
 * two sides' traces averaged; face point indexed by the two other node
 * indices, lower axis fastest).  Buffers are host memory owned by the caller.
 * Errors: BGK_EINVAL (missing arguments, invalid sizes, a non-positive
 * Jacobian). */
BGK_API bgk_status bgk_curved_metrics(const bgk_mesh_desc *mesh, double *S, double *J, double *fvec);

/* The 1-D FR operators the library builds for order p (host only, section
 * "Numerical method": Gauss--Legendre nodes, the Lagrange derivative, the
 * traces l_j(+-1), the DG-recovering correction-function derivatives), q =
 * p + 1: fr_out = [xi(q), w(q), D(q*q, row-major D_ij = l_j'(xi_i)), l(-1)(q),
 * l(+1)(q), g_L'(q), g_R'(q)]; and the FP32 tables of the curvilinear mixed
 * stage: curv32_out = [D(q*q), l(+1)(q), l(-1)(q), g_L'(q), g_R'(q), def(q)]
 * (l(-1) and g_L' the mirror images of l(+1) and g_R', def the column-sum
 * defects of the rounded deviation-form operator divided by sum w).  Buffers
 * are host memory owned by the caller.  Errors: BGK_EINVAL. */
BGK_API bgk_status bgk_fr_tables(int order, double *fr_out, float *curv32_out);

/* N_e, N_s, N_u and the number of components (1 or 2); any output may be
 * NULL.  Errors: BGK_EINVAL (NULL context). */
BGK_API bgk_status bgk_sizes(const bgk_ctx *ctx, int *n_elem, int *n_sol, int *n_vel, int *n_comp);

/* Solution-node coordinates x[P][3], P = N_e N_s: on the uniform box in the
 * context's own Gauss--Legendre node placement; on a curvilinear mesh the
 * node_xyz the context was created with.  x is host (on_device = 0) or device
 * memory (1), written before the call returns.  Errors: BGK_EINVAL, BGK_ECUDA. */
BGK_API bgk_status bgk_node_coords(const bgk_ctx *ctx, double *x, int on_device);

/* Copy the state in / out: the distribution f of section "Governing
 * equations" (F, and G when delta > 0) as f[c][k][e][s], double for
 * BGK_FP64 and float for BGK_MIXED, C N_u P elements.  f is host
 * (on_device = 0) or device memory (1); host copies complete before the
 * call returns, device copies are ordered on the context's stream.  Setting
 * the state invalidates the cached moments.  Errors: BGK_EINVAL (NULL),
 * BGK_ECUDA. */
BGK_API bgk_status bgk_set_state(bgk_ctx *ctx, const void *f, int on_device);
BGK_API bgk_status bgk_get_state(bgk_ctx *ctx, void *f, int on_device);

/* Set f to the isotropic Maxwellian of q[P][5] = (rho, U1, U2, U3, theta) at
 * every node (G = delta theta / 2 F).  Section "Governing equations", g_u
 * with T = theta I.  q is host (on_device = 0) or device memory (1).
 * Errors: BGK_EINVAL (NULL), BGK_ECUDA. */
BGK_API bgk_status bgk_set_maxwellian(bgk_ctx *ctx, const double *q, int on_device);

/* Run bgk_step as CUDA-graph replays (enable = 1) or as direct launches
 * (0, the default).  With graphs on, the first step captures the six
 * launches of one SSP-RK3 step (Q' solve and fused stage, three times) into a
 * graph per buffer parity and later steps replay it; a graph is captured
 * again whenever something baked into its kernel arguments changes (dt, the
 * Newton settings, the learned-guess mode, the training log, the stage
 * kernel).  Results are bit-identical to direct launches.  While profiling
 * (bgk_profile) is on, steps run as direct launches so each kernel can be
 * timed.  Errors: BGK_EINVAL, BGK_ECUDA.  The paper's method has no notion
 * of graphs; this is the launch mechanism only. */
BGK_API bgk_status bgk_set_graphs(bgk_ctx *ctx, int enable);

/* Tensor variant of the discrete ES equilibrium (section "Numerical method":
 * ES-BGK may need a nonlinear solve of marginally higher dimension when the
 * velocity grid lacks symmetry).  enable = 1: after the d+2 solve, each
 * point's equilibrium is refined to the discrete Gaussian
 * exp(b . phi(u - U)), phi = (1, u - U, (u_i - U_i)(u_j - U_j), i <= j), whose
 * discrete moments are (rho, 0, rho T) with T = theta/Pr I + (1 - 1/Pr) Pi/rho
 * the ES target: ten unknowns, Newton on b (symmetric positive definite
 * Jacobian, unique solution).  Mass, momentum and energy stay conserved and
 * the discrete stress of the equilibrium is rho T exactly (the d+2 solve
 * matches only its trace).  The Newton statistics (bgk_stats) then count the
 * refinement's updates; no training pairs are logged.  bgk_qprime keeps
 * returning the d+2 solution.  Default 0.
 * Errors: BGK_EINVAL; BGK_ENOTSUP for delta > 0 (a reading for the
 * monatomic gas only). */
BGK_API bgk_status bgk_set_es_tensor(bgk_ctx *ctx, int enable);

/* Newton controls of the Q' solve (section "Numerical method": Newton's
 * method on the discrete compatibility conditions): stop when the scaled
 * residual max(|R_rho|/rho, |R_rhoU|_inf/(rho sqrt(theta)), |R_E|/E) <= tol,
 * at most max_iter updates (defaults 1e-13, 50).  Errors: BGK_EINVAL (NULL,
 * tol not positive, max_iter < 0). */
BGK_API bgk_status bgk_set_newton(bgk_ctx *ctx, double tol, int max_iter);

/* Engine of the Q' velocity sums (the discrete compatibility solve of
 * section "Numerical method"; the result is the same solution, the engine
 * only sets the arithmetic of its sums).  fp32_sums = 0: FP64 throughout (the FP64
 * form, and optionally the mixed form).  fp32_sums = 1 (mixed form only, its
 * default): the velocity sums of the Newton iteration run on the FP32 pipe
 * (GB300 issues FP64 at 1/64 of the FP32 rate), the per-point Newton algebra
 * in FP64, stopping at a scaled residual of 1e-6; the discrete compatibility
 * of the equilibrium actually used is then restored by the FP32-equilibrium
 * moment correction, which measures its moments with exact compensated sums
 * against the moments of f.  Errors: BGK_EINVAL for fp32_sums on the FP64 form. */
BGK_API bgk_status bgk_set_qprime_engine(bgk_ctx *ctx, int fp32_sums);

/* Kernel of the mixed-form stage (the fused step of section "Methodology":
 * FR advection, BGK source, Runge--Kutta update and the moments of the
 * result).  All variants compute the same values bit for bit.
 *   0 (default) the asynchronous-copy kernel where it applies, else the plain one;
 *   1 plain: each thread loads its operands itself, one block-wide barrier
 *     per velocity;
 *   2 async: a producer warp stages the element run, its upwind neighbours
 *     and f^n for up to `depth` velocities ahead with bulk copies completing
 *     on mbarriers; one thread per solution node;
 *   3 line: the same copy ring, one thread per first-axis node line (p + 1
 *     points), short element runs;
 *   4 line, runs twice as long;
 *   5 half: the same copy ring, one thread per half first-axis node line;
 *   6 half, runs twice as long.
 * depth: 2..16 copy-ring stages (default 6).  Variants 2-6 need p = 1 or 3
 * (element slabs of whole 16-byte units) and 16-byte aligned state buffers
 * (bgk_stage runs caller buffers that are not on the plain kernel); every
 * wait in them is bounded and a wait that gives up makes the next status
 * check return BGK_ETIMEOUT.  Errors: BGK_EINVAL (range), BGK_ENOTSUP
 * (variants 2-6 on the FP64 form or an unsupported order). */
BGK_API bgk_status bgk_set_stage_kernel(bgk_ctx *ctx, int variant, int depth);

/* Velocity blocking of the stage and moment kernels: the velocities are
 * split into n blocks of whole first-axis lines (the last may be shorter),
 * each a separate CTA column of the stage grid with its own moment partials
 * (bgk_create picks about enough blocks to fill the GPU; more blocks fill its
 * last wave of CTAs better and cost the Q' solve more partial sums;
 * bgk_tune_stage also chooses n).  The values computed change in the last
 * bits with n (the partial sums are taken in another grouping), not beyond.
 * Waits for the context's stream; the next step recomputes the moments.
 * Errors: BGK_EINVAL (NULL, n < 1, n above the context's maximum, given by
 * bgk_get_velocity_blocks). */
BGK_API bgk_status bgk_set_velocity_blocks(bgk_ctx *ctx, int n);
/* The current velocity blocking: number of blocks, velocities per block and
 * the most blocks bgk_set_velocity_blocks accepts (outputs may be NULL).
 * Errors: BGK_EINVAL (NULL context). */
BGK_API bgk_status bgk_get_velocity_blocks(const bgk_ctx *ctx, int *n_blocks, int *per_block, int *max_blocks);

/* Test entry for the bounded waits of the copy-ring kernels (variants 2-6):
 * with after > 0 every block's ring delivers only its first `after`
 * velocities and stops, so the consumers' next wait runs out, after
 * wait_seconds (0: about 2 s) instead of about 2 s; the kernel then lets its
 * issued copies land, sets its timeout status and returns, and the next
 * status check reports BGK_ETIMEOUT.  The state written by such a stage is
 * incomplete.  after = 0 restores normal operation (and the 2 s limit).
 * Waits for the context's stream first.  Errors: BGK_EINVAL (NULL, after < 0,
 * wait_seconds outside [0, 10]). */
BGK_API bgk_status bgk_test_ring_stall(bgk_ctx *ctx, int after, double wait_seconds);

/* Autotune the mixed-form stage kernel on this context's own problem (the
 * launch configuration only; every kernel candidate computes the same values):
 * time the plain kernel and every supported asynchronous variant at every ring
 * depth (2, 3, 4, 6, 8, 12, 16), each over `reps` stages with f^n and the moment
 * epilogue (time step dt), from the current state into a scratch buffer, and
 * keep the fastest (as bgk_set_stage_kernel would); then, for that kernel, time
 * Q' solve + stage at the velocity blockings from the current count to four
 * times it that split the lines evenly and keep the fastest (as
 * bgk_set_velocity_blocks would); then, at that blocking, time the kernel's
 * ring depths again and keep the fastest.  The state is not
 * changed; the cached moments are recomputed by the next step.  Outputs (each
 * may be NULL): the chosen variant and depth and its mean time per stage in
 * ms (at the chosen blocking; for the plain kernel at the default one).  The FP64 form has one kernel: only its velocity blocking is chosen (by
 * the stage's time); returns variant 1 and that kernel's time.  Errors:
 * BGK_EINVAL, BGK_ECUDA, BGK_ETIMEOUT, BGK_ENOCONV (the Q' solve of the
 * current state). */
BGK_API bgk_status bgk_tune_stage(bgk_ctx *ctx, double dt, int reps, int *variant_out, int *depth_out,
                                  double *ms_out);

/* One residual R(f) = -div(u f) + (g(Q') - f)/tau of f_in into r_out (the
 * semi-discrete right-hand side of section "Methodology": FR advection plus
 * the conservative BGK source), both with the state's layout and element
 * type, both host (on_device = 0) or both device memory (1).  Test and debug
 * entry; it leaves the state unchanged.  Errors: BGK_EINVAL (NULL), BGK_ECUDA,
 * BGK_ENOCONV (a Q' solve did not converge; r_out uses the last iterate). */
BGK_API bgk_status bgk_rhs(bgk_ctx *ctx, const void *f_in, void *r_out, int on_device);

/* Pipelined stepping from host memory to host memory: copy the state f_in
 * (host, layout of bgk_set_state) to the device, advance it n_steps SSP-RK3
 * steps of size dt, copy the result to f_out (host).  Asynchronous: the call
 * returns after enqueueing; the host-to-device copy of this call and the
 * device-to-host copy of the previous call's result run on their own streams
 * and overlap the compute, so a loop of calls keeps both copy directions and
 * the GPU busy at once.  f_in and f_out must stay valid and unmodified until
 * bgk_step_host_sync returns (pinned memory gives the full copy rate).  Uses
 * one or two more state-sized device buffers (allocated on the first call;
 * two when the device has 8 GiB to spare beyond them, so that an input copy
 * waits only for the output copy of three calls back) and direct launches
 * instead of CUDA graphs.  Any other call that reads or writes the
 * state waits for the pipeline first.  Errors: BGK_EINVAL (NULL, dt <= 0,
 * n_steps < 1), BGK_ENOTSUP (a velocity shard), BGK_ENOMEM, BGK_ECUDA. */
BGK_API bgk_status bgk_step_host(bgk_ctx *ctx, const void *f_in, void *f_out, double dt, int n_steps);
/* Wait for every bgk_step_host call: all results are in their f_out, the
 * context's state is the last result.  Device failures (Newton
 * non-convergence, a bounded wait that gave up) are reported here.  Errors:
 * BGK_EINVAL (NULL), BGK_ENOCONV, BGK_ETIMEOUT, BGK_ECUDA. */
BGK_API bgk_status bgk_step_host_sync(bgk_ctx *ctx);

/* n_steps steps of SSP-RK3 (Shu--Osher) with step dt on the stored state
 * (the explicit time marching of section "Methodology").  Each stage is two
 * kernels: the Q' solve from the moments of the stage input, and the fused
 * FR + source + RK update that also reduces the moments of its output.
 * n_steps = 0 leaves the state as it is.  Errors: BGK_EINVAL (NULL, dt not
 * positive, n_steps < 0), BGK_ECUDA, BGK_ETIMEOUT; BGK_ENOCONV if a Newton
 * solve did not converge (the step is still completed with the last
 * iterate). */
BGK_API bgk_status bgk_step(bgk_ctx *ctx, double dt, int n_steps);

/* One Shu--Osher stage f_out = a f^n + b f_s + c R(f_s) with f^n = f_n (may
 * be NULL when a = 0) and f_s = f_in: device arrays in the state's layout
 * and element type; f_out must not alias f_in.  The stored state is not
 * used or changed.  Errors: BGK_EINVAL (NULL f_in or f_out, aliasing, a != 0
 * without f_n), BGK_ECUDA, BGK_ETIMEOUT, BGK_ENOCONV. */
BGK_API bgk_status bgk_stage(bgk_ctx *ctx, const void *f_n, const void *f_in, void *f_out,
                     double a, double b, double c);

/* Raw velocity moments of the stored state (section "Governing equations":
 * the moments that give Q = (rho, rho U, E)), m[P][11]: sum w F, sum w u_d F
 * (3), sum w u_d^2 F (3), sum w u1u2 F, sum w u1u3 F, sum w u2u3 F, sum w G,
 * summed in FP64.  m is host (on_device = 0) or device memory (1).
 * Errors: BGK_EINVAL (NULL), BGK_ECUDA. */
BGK_API bgk_status bgk_moments(bgk_ctx *ctx, double *m, int on_device);

/* Raw moments of a caller-owned state without allocating any device memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc (a framework that has claimed the whole memory
 * pool, a real-time loop that must not allocate, a plugin host that forbids
 * allocation) and therefore cannot create a context.
 *   vgrid   velocity grid (as for bgk_create); N_u = n[0] n[1] n[2]
 *   f       device array f[n_comp][N_u][n_points], double (BGK_FP64 layout)
 *   m       device output m[n_points][11], slots as in bgk_moments
 *   stream  cudaStream_t (NULL = legacy default stream); the call is
 *           asynchronous on it and returns after the launches.
 * Scratch: a fixed 16 MiB device array inside libbgk (2^21 doubles), held by
 * every GPU that loads the library until the process exits;
 * n_points * 11 must not exceed 2^21 (n_points <= 190650), else BGK_EINVAL.
 * All calls share that array, so calls that overlap on the GPU race; each
 * call overwrites every partial sum it reads, so nothing needs clearing.
 * The array's device address belongs to a CUDA context: a call whose stream
 * is not being captured looks it up for the context current on the calling
 * thread (the first such call on a device is the set-up), so calls from
 * another context on the same device, or after cudaDeviceReset, use their
 * own context's copy.  A call made while its stream is being captured reuses
 * the address found by the last uncaptured call on that device (BGK_ECUDA if
 * there was none): make one call, from the capturing context, before any
 * stream capture.  Errors: BGK_EINVAL, BGK_ECUDA. */
BGK_API bgk_status bgk_moments_noalloc(const bgk_vgrid_desc *vgrid, const double *f, int n_comp,
                                       int n_points, double *m, void *stream);

/* Macroscopic fields of the current state per solution point (section
 * "Results": the density gradient-length local Knudsen number
 * Kn_GLL = lambda ||grad rho||_2 / rho with the local mean free path
 * lambda = (mu(theta)/rho) sqrt(pi/(2 theta)); continuum breakdown is expected
 * above 0.05), out[n_elem * n_sol][10] FP64, points e-major:
 *   rho, U1, U2, U3, theta, p, Mach = |U|/sqrt(gamma theta), lambda,
 *   ||grad rho||_2, Kn_GLL.
 * grad rho is the gradient of the FR-corrected density polynomial (nodal
 * derivative plus correction-function terms carrying the central common
 * interface value; at a Dirichlet face the average with the face state's
 * density; at a specular, diffuse or collapsed face the element's own trace);
 * on a curvilinear mesh by the chain rule through the metric terms,
 * grad rho = (1/J) sum_d S^d d rho/d xi_d.  out is host memory
 * (on_device = 0) or device memory (1).  Errors: BGK_EINVAL, BGK_ECUDA;
 * BGK_ENOTSUP on a velocity shard (the moments would be partial). */
BGK_API bgk_status bgk_macro(bgk_ctx *ctx, double *out, int on_device);

/* The Q' solve alone (section "Numerical method", discrete compatibility):
 * from raw moments m[n_points][11] (layout of bgk_moments) to
 * qp[n_points][5] = (rho', U'_1..3, theta') and Newton update counts
 * iters[n_points] (may be NULL).  Returns BGK_ENOCONV if any point failed. */
BGK_API bgk_status bgk_qprime(bgk_ctx *ctx, const double *m, int n_points, double *qp, int *iters,
                      int on_device);

/* ---- Velocity shards (several GPUs, one per shard) -------------------------
 * The method couples velocities only through the moments of f (section
 * "Numerical method": the FR advection of every velocity is independent, the
 * BGK source needs Q of the whole velocity set).  So the velocity set can be
 * split: a shard holds the third-axis velocity planes [slab_lo, slab_hi) of
 * the grid for every element and node, and one SSP-RK3 step is three rounds of
 *   bgk_shard_partials(shard, m)      partial raw moments of the stage input
 *   (the caller sums m over all shards, e.g. an NCCL all-reduce, in place)
 *   bgk_shard_stage(shard, m, stage, dt)   Q' from the summed moments over the
 *                                     whole grid, then the fused stage on the
 *                                     shard's own velocities
 * for stage = 0, 1, 2.  Every shard solves Q' for every point (the same
 * inputs give the same q' everywhere); the exchange is 11 doubles per point
 * per stage.  The shards of one grid together equal the unsharded context.
 *
 * bgk_create_shard: as bgk_create, vgrid describing the WHOLE grid; the
 * context holds n[0] n[1] (slab_hi - slab_lo) velocities (bgk_sizes), in the
 * layout of bgk_set_state with the third axis restricted to the slab.
 * Trapezoid weights are those of the whole grid (half weight only at its
 * ends).  Supported: periodic and Dirichlet faces on box or curvilinear
 * meshes.  Errors: BGK_EINVAL (slab outside [0, n[2]] or fewer than two
 * planes, and bgk_create's checks), BGK_ENOTSUP (specular, diffuse or closed
 * faces), BGK_ENOMEM, BGK_ECUDA.  On a shard bgk_moments and bgk_totals
 * return the shard's part (sums over its velocities; add them over the
 * shards); bgk_step, bgk_stage, bgk_rhs, bgk_macro and bgk_tune_stage return
 * BGK_ENOTSUP. */
BGK_API bgk_status bgk_create_shard(bgk_ctx **out, const bgk_mesh_desc *mesh, const bgk_vgrid_desc *vgrid,
                                    const bgk_gas_desc *gas, int precision, void *cuda_stream, int slab_lo,
                                    int slab_hi);
/* Partial raw moments of the current stage input over this context's
 * velocities, m[11][n_points] FP64 in DEVICE memory (caller-owned; slot order
 * of bgk_moments, transposed: slot-major), written asynchronously on the
 * context's stream.  Also valid on an unsharded context (then the full
 * moments).  Errors: BGK_EINVAL (NULL), BGK_ECUDA. */
BGK_API bgk_status bgk_shard_partials(bgk_ctx *ctx, double *m);
/* Stage `stage` (0, 1, 2) of an SSP-RK3 step of size dt from the moments m
 * (device [11][n_points], summed over all shards of the grid): the Q' solve
 * over the whole grid, the fused stage on this context's velocities, and the
 * partial moments of the next stage's input; after stage 2 the stored state
 * is the step's result.  Asynchronous apart from the device status read.
 * Errors: BGK_EINVAL (NULL, stage or dt out of range, no partials taken
 * since the state was set), BGK_ENOCONV, BGK_ETIMEOUT, BGK_ECUDA. */
BGK_API bgk_status bgk_shard_stage(bgk_ctx *ctx, const double *m, int stage, double dt);

/* Domain totals (rho, rho U, E) = sum_e sum_s W_s J_s sum_k w_k psi_k f of
 * the stored state (W_s tensor Gauss weights, J_s the Jacobian at the node:
 * the affine |J_e| on the box; on a curvilinear mesh det(dX/dxi) of the
 * element's interpolant in the FP64 form, and 1 / (1/J_s rounded to FP32) in
 * the mixed form, the quadrature its stage conserves exactly): the conserved
 * quantities of section "Governing equations".  totals is host memory.
 * entropy (host memory, may be NULL): the discrete entropy
 * H = sum_e sum_s W_s J_s sum_k w_k F ln F of the stored F component with the
 * same quadrature, summed in FP64 (section "Numerical method": the
 * discrete-velocity BGK relaxation does not increase it).  It is NaN when
 * some stored F is not positive.  With delta > 0 it covers F only (the paper
 * states no entropy functional for the reduced F, G pair).
 * Errors: BGK_EINVAL (NULL context or totals), BGK_ECUDA. */
BGK_API bgk_status bgk_totals(bgk_ctx *ctx, double totals[5], double *entropy);

/* Newton statistics accumulated since the last call (then reset):
 * mean and max update count per point solve, and the worst final scaled
 * residual; any output may be NULL.  Errors: BGK_EINVAL (NULL context),
 * BGK_ECUDA. */
BGK_API bgk_status bgk_stats(bgk_ctx *ctx, double *mean_iters, int *max_iters, double *max_residual);

/* Per-kernel timing on the context's stream (instrumentation; the paper has
 * no counterpart).  enable = 1 starts recording a
 * CUDA event pair around every kernel the context launches (and clears the
 * accumulators); 0 stops.  bgk_profile_read synchronises and returns, per
 * kernel kind (BGK_K_*), the summed device milliseconds and launch counts
 * since the last enable; either array may be NULL (host memory otherwise).
 * Launch counts are kept even when timing is off.  Errors: BGK_EINVAL (NULL
 * context), BGK_ECUDA. */
#define BGK_K_MOMENTS 0    /* raw moment partials of a state            */
#define BGK_K_QPRIME 1     /* moment reduction + Q' Newton solve        */
#define BGK_K_STAGE 2      /* fused FR + source + RK + moment epilogue  */
#define BGK_K_OTHER 3      /* initialisation and reductions             */
#define BGK_K_WALL 4       /* diffuse-wall densities of a stage's input  */
#define BGK_NKINDS 5
BGK_API bgk_status bgk_profile(bgk_ctx *ctx, int enable);
BGK_API bgk_status bgk_profile_read(bgk_ctx *ctx, double ms[BGK_NKINDS], long long launches[BGK_NKINDS]);

/* Roofline probes of the current device (no context; measurement, not the
 * method): kind 0 = FP64 FMA throughput, 1 = FP32 FMA throughput (both in
 * flop/s, an FMA = 2 flops), 2 = FP64 exp() throughput (calls/s), 3 = FP32
 * exp2f throughput (calls/s), into *value (host).  Each runs a
 * register-resident kernel over every SM for ~50 ms.  Errors: BGK_EINVAL
 * (kind out of range, NULL value), BGK_ENOMEM, BGK_ECUDA. */
BGK_API bgk_status bgk_probe_peak(int kind, double *value);

/* Tensor-core probe of the FR element operator at p = 3 (no context;
 * measurement, not the method's path).  Per direction the FR derivative of
 * one element at one velocity, with the own-trace lift folded in, is a dense
 * 64 x 64 operator on the element's nodes (section "Numerical method"); this
 * streams n_panels panels of 48 element-velocity columns (BF16 hi and lo
 * parts of FP32 data, 12 KB each, generated on the device and read by TMA
 * tiled copies) through tcgen05 MMAs (BF16 x 3 split products, FP32
 * accumulation in tensor memory) for all three directions and reads the
 * accumulators back, then checks 8 seeded panels against FP64 on the host.
 * out (host): [0] useful MMA flop/s, [1] element-node-velocity operator
 * applications (DOF, three directions each) per second, [2] operand bytes
 * streamed per second, [3] largest error of an output relative to the sum of
 * its terms' magnitudes, [4] relative bias of the outputs' magnitudes
 * (negative: shrunk toward zero), [5] kernel milliseconds.  Allocates
 * n_panels x 12 KB of device memory for the call.  Errors: BGK_EINVAL
 * (n_panels outside [16, 2^22], NULL out), BGK_ENOTSUP (not an sm_103
 * device, or no tensor-map encoder), BGK_ENOMEM, BGK_ECUDA, BGK_ETIMEOUT (a
 * bounded wait in the kernel gave up). */
BGK_API bgk_status bgk_probe_tc(long long n_panels, double out[6]);

/* ---- Learned initial guess of the Q' solve -------------------------------
 * Not in the paper (which starts Newton from the macroscopic state): a
 * 9 -> 64 -> 64 -> 5 SiLU network maps the point's state to a correction
 * Delta whose application gives Newton's starting point, trained on the GPU
 * on pairs logged by the solver's own converged solves.  Features: rho,
 * U1..3, theta, the invariants tr A, (tr(A)^2 - tr(A^2))/2, det A of
 * A = Pi/(rho theta), and the mean free path lambda = mu/rho sqrt(pi/(2 theta)).
 * Target: rho'/rho - 1, (U' - U)/sqrt(theta), theta'/theta - 1.  Weights and
 * layer inputs are rounded to BF16 (bf16 = 1), sums accumulate in FP32, the
 * optimiser (Adam) keeps FP32 master weights.  A guess whose first scaled
 * residual exceeds 1e-3, or from which Newton does not converge, is
 * discarded and the solve restarts from the macroscopic state. */
#define BGK_MLP_NPARAM 5125   /* W1[9][64] b1[64] W2[64][64] b2[64] W3[64][5] b3[5] */
#define BGK_MLP_NNORM 28      /* x_mean[9] x_std[9] t_mean[5] t_std[5] */
#define BGK_MLP_LOG_STRIDE 14 /* 9 features then 5 targets per logged pair */

/* mode 0: start Newton from the macroscopic state; 1: from the network
 * (requires weights from bgk_mlp_train or bgk_mlp_weights); bf16 = 1 runs
 * the inference on BF16-rounded weights and layer inputs.  Errors:
 * BGK_EINVAL (NULL, mode out of range, mode 1 without weights). */
BGK_API bgk_status bgk_set_guess(bgk_ctx *ctx, int mode, int bf16);
/* Start (enable = 1, clearing earlier pairs) or stop logging the (features,
 * Delta) pair of every converged point solve, at most max_pairs of them
 * (device memory owned by the context).  Errors: BGK_EINVAL (NULL, enable
 * with max_pairs <= 0), BGK_ENOMEM, BGK_ECUDA. */
BGK_API bgk_status bgk_mlp_log(bgk_ctx *ctx, int enable, long long max_pairs);
/* Copy up to max_pairs logged pairs (host out[n][14]); *n_out = pairs copied.
 * Errors: BGK_EINVAL (NULL, max_pairs < 0), BGK_ECUDA. */
BGK_API bgk_status bgk_mlp_log_read(bgk_ctx *ctx, float *out, long long max_pairs, long long *n_out);
/* Train from scratch on the logged pairs: normalisation from their mean and
 * standard deviation, He-normal initialisation from seed, Adam with a cosine
 * learning-rate decay from lr to lr/10, MSE loss on normalised targets.
 * *final_loss (host, may be NULL) = mean batch loss of the last epoch.
 * Errors: BGK_EINVAL (NULL, epochs, batch or lr not positive, fewer logged
 * pairs than one batch), BGK_ENOMEM, BGK_ECUDA. */
BGK_API bgk_status bgk_mlp_train(bgk_ctx *ctx, int epochs, int batch, float lr, unsigned long long seed,
                                 int bf16, double *final_loss);
/* Save (load = 0) or load (load = 1) the weights and normalisation:
 * host buf[BGK_MLP_NPARAM + BGK_MLP_NNORM], copied.  Errors: BGK_EINVAL
 * (NULL, saving before any training or load), BGK_ECUDA. */
BGK_API bgk_status bgk_mlp_weights(bgk_ctx *ctx, float *buf, int load);
/* Loss and gradient of the current weights on one batch (host arrays:
 * x[n][9] raw features, t[n][5] raw targets, grad[BGK_MLP_NPARAM]); the
 * training kernel's forward and backward pass without the update.  Errors:
 * BGK_EINVAL (NULL, n <= 0, no trained or loaded network), BGK_ENOMEM,
 * BGK_ECUDA. */
BGK_API bgk_status bgk_mlp_grad(bgk_ctx *ctx, const float *x, const float *t, int n, int bf16, double *loss,
                                float *grad);
/* Batched inference of the current network on tensor cores: the guess
 * correction delta[n][5] for raw features x[n][9] (layouts of the training
 * pairs), BF16 weights and layer inputs, FP32 accumulation in tensor memory
 * (tcgen05), FP32 biases and SiLU; the same network the Newton kernel
 * evaluates inline for every point.  x and delta are device (on_device = 1)
 * or host memory.  Errors: BGK_EINVAL (NULL, n outside [1, 2^31], no trained
 * or loaded network), BGK_ENOMEM, BGK_ECUDA, BGK_ETIMEOUT (a bounded wait in
 * the kernel gave up). */
BGK_API bgk_status bgk_mlp_infer(bgk_ctx *ctx, const float *x, long long n, float *delta, int on_device);
/* Number of learned guesses discarded since the last call (then reset), into
 * host *fallbacks.  Errors: BGK_EINVAL (NULL), BGK_ECUDA. */
BGK_API bgk_status bgk_mlp_stats(bgk_ctx *ctx, unsigned long long *fallbacks);

/* Text of the last error on this context (never NULL; "null context" for a
 * NULL context); valid until the next call on the context. */
BGK_API const char *bgk_last_error(const bgk_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* BGK_H */
