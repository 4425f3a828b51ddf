/*
 * dg.h -- C ABI of the GB300 matrix-free discontinuous Galerkin solver for the
 * first-order acoustic wave equation (Schoeder, Kormann, Wall, Kronbichler,
 * "Efficient Explicit Time Stepping of High Order Discontinuous Galerkin
 * Schemes for Waves").
 *
 * Problem (Sec. 2, Eq. (1)): du/dt + S u = 0 with u = (p, v),
 *   dv/dt + rho^-1 grad p = 0,   dp/dt + rho c^2 div v = 0.
 * Discretisation (Sec. 2.1, Eqs. (2)-(3)): DG on hexahedra, tensor degree k,
 * state stored in the Lagrange basis on the (k+1)^3 Gauss-Lobatto nodes
 * ("GL", Sec. 3.1), integrals by (k+1)^3 / (k+1)^2 Gauss points, mass terms
 * weighted by rho (velocity) and 1/(rho c^2) (pressure); upwind (alpha = 1)
 * or central (alpha = 0) impedance-weighted flux (Sec. 2.4).
 *
 * Conventions
 * -----------
 * - Every call returns an int status (DG_OK = 0, negative = error). No call
 *   aborts, throws or exits; on error the context (when one is given) keeps
 *   a message readable through dg_last_error().
 * - State layout: U[E][4][(k+1)^3], fields (p, v_x, v_y, v_z), nodes
 *   lexicographic with the first reference axis fastest. Element-local node
 *   values in the GL basis. Device states are caller-owned device pointers in
 *   the context's precision (double for DG_FP64, float for DG_FP32), 16-byte
 *   aligned (DG_EINVAL otherwise).
 * - Streams are passed as uintptr_t holding a cudaStream_t (0 = legacy
 *   default stream). All device work of a call is enqueued on that stream;
 *   calls return once the work is enqueued unless stated otherwise.
 * - Host arrays passed in are caller-owned and only read during the call.
 * - Contexts are not thread safe: one thread at a time per context.
 */
#ifndef DG_H
#define DG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define DG_OK            0
#define DG_EINVAL       -1  /* bad argument (NULL, size, range) */
#define DG_ENOMEM       -2  /* device or host allocation failed */
#define DG_ECUDA        -3  /* a CUDA runtime call failed */
#define DG_EUNSUPPORTED -4  /* e.g. degree outside [1, DG_KMAX] */
#define DG_EAGAIN       -5  /* dg_poll: request not finished yet */
#define DG_ETIMEOUT     -6  /* a bounded device wait gave up */
#define DG_EMESH        -7  /* inconsistent connectivity or det J <= 0 */

/* precisions */
#define DG_FP64 0  /* operator, state and geometry in double */
#define DG_FP32 1  /* operator and state in float; geometry set up in double */

#define DG_KMAX 7

typedef struct dg_ctx dg_ctx;

/*
 * Mesh description (all host arrays, caller-owned, read during the call).
 *  n_elem       number of hexahedra E >= 1
 *  geom_degree  q >= 1: each element is the image of [-1,1]^3 under the
 *               degree-q Lagrange interpolant of its geometry nodes
 *  nodes        [E][(q+1)^3][3] physical positions of the geometry nodes at
 *               the tensor Gauss-Lobatto points of degree q (first axis
 *               fastest)
 *  nbr          [E][6] neighbour element across local face f, or -1 for a
 *               reflecting wall. Faces: 0 -xi, 1 +xi, 2 -eta, 3 +eta,
 *               4 -zeta, 5 +zeta. Periodicity is expressed by nbr alone.
 *  nbr_face     [E][6] the neighbour's local face index (ignored at walls)
 *  orient       [E][6] orientation code 0..7. The tangential axes of face f
 *               are the two reference axes other than f/2, in increasing
 *               order; a face point has indices (i, j) along them. Code o
 *               maps (i, j) to the neighbour's (i', j'): (u, v) = (j, i) if
 *               o & 1 else (i, j); i' = n-1-u if o & 2 else u;
 *               j' = n-1-v if o & 4 else v.
 */
typedef struct {
  int32_t n_elem;
  int32_t geom_degree;
  const double* nodes;
  const int32_t* nbr;
  const int8_t* nbr_face;
  const int8_t* orient;
} dg_mesh_desc;

/*
 * Validate the mesh (index ranges, nbr/nbr_face symmetry, orientation codes
 * that are mutual inverses), upload it, compute geometry in FP64 on the GPU
 * (inverse Jacobians, determinants, face normals; Sec. 3 "pre-computed
 * inverse Jacobians", Sec. 3.3) with rho = c = 1, and return a context.
 *  k           polynomial degree, 1 <= k <= DG_KMAX
 *  prec        DG_FP64 or DG_FP32
 *  flux_alpha  1 = upwind (HDG flux with tau = 1/(rho c), Sec. 2.4),
 *              0 = central; any value in [0, 1]
 *  stream      stream for the set-up work; the call synchronises it
 * Errors: DG_EINVAL, DG_EUNSUPPORTED, DG_EMESH (bad connectivity or a
 * non-positive Jacobian determinant anywhere), DG_ENOMEM, DG_ECUDA.
 * On error *out is NULL and nothing is leaked.
 */
int dg_mesh_setup(const dg_mesh_desc* mesh, int k, int prec, double flux_alpha,
                  uintptr_t stream, dg_ctx** out);

/*
 * dg_mesh_setup with the coefficients given at once (rho, c as for
 * dg_set_coefficients), so the geometry set-up runs once. rho and c are both
 * NULL (rho = c = 1) or both given.
 */
int dg_mesh_setup_coef(const dg_mesh_desc* mesh, int k, int prec, double flux_alpha,
                       const double* rho, const double* c, uintptr_t stream, dg_ctx** out);

/*
 * 2D meshes of quadrilaterals (the paper treats d = 2 and d = 3 alike,
 * Sec. 2; its 2D experiments are in Sec. 4.7). Faces 0: xi = -1, 1: xi = +1,
 * 2: eta = -1, 3: eta = +1; node (x, y) of an element at x + n y.
 *   nodes    [E][(q+1)^2][2]  GL geometry nodes
 *   nbr      [E][4]           neighbour across face f, -1 = wall
 *   nbr_face [E][4]           the neighbour's face
 *   orient   [E][4]           1 when the neighbour's face coordinate runs
 *                             opposite to this element's, else 0; must be
 *                             reciprocated
 * rho, c: [E][(k+1)^2] at the GL solution nodes, or both NULL (= 1).
 * States are [E][3][(k+1)^2] (p, v_x, v_y), GL nodal values, 16-byte
 * aligned. A 2D context steps with the state in the Gauss basis (dg_set_basis
 * accepts DG_BASIS_G only) and takes dg_apply_operator, dg_step_lsrk,
 * dg_step_ader (reduce_every 0 or 2), dg_tck, dg_energy, dg_norms,
 * dg_solve_host, dg_set_coefficients, dg_change_basis and the query and
 * profiling calls. Batches, parts, the server, tuning, HDG-ADER and
 * dg_energy_noalloc return DG_EUNSUPPORTED for it. Errors as dg_mesh_setup.
 */
typedef struct {
  int32_t n_elem;
  int32_t geom_degree;
  const double* nodes;
  const int32_t* nbr;
  const int8_t* nbr_face;
  const int8_t* orient;
} dg_mesh2d_desc;
int dg_mesh_setup_2d(const dg_mesh2d_desc* mesh, int k, int prec, double flux_alpha, const double* rho,
                     const double* c, uintptr_t stream, dg_ctx** out);

/*
 * Set the coefficients rho > 0 and c > 0 (Sec. 2, Eq. (1)) as host arrays
 * [E][(k+1)^3] of values at each element's GL solution nodes; each is the
 * degree-k polynomial through those values, and may jump between elements.
 * Recomputes mass diagonals, impedances and predictor coefficients in FP64.
 * Synchronises the stream. Errors: DG_EINVAL (NULL, non-positive value),
 * DG_ECUDA.
 */
int dg_set_coefficients(dg_ctx* ctx, const double* rho, const double* c,
                        uintptr_t stream);

/*
 * R = -M^-1 K U (Sec. 2.1 Eq. (3)): the semi-discrete right-hand side,
 * cell terms by sum factorisation at Gauss points, face fluxes from the GL
 * face nodes of both neighbours (Sec. 3.1), inverse mass by the basis change
 * GL -> G, diagonal, G -> GL (Sec. 3.1). U and R are device arrays
 * [E][4][(k+1)^3] that must not overlap.
 */
int dg_apply_operator(dg_ctx* ctx, const void* U, void* R, uintptr_t stream);

/*
 * nsteps of the five-stage fourth-order 2N-storage low-storage Runge-Kutta
 * scheme (Sec. 2.2), dU <- A_s dU + dt R(U); U <- U + B_s dU, with the vector
 * updates fused into the operator kernel. U (device) holds the initial state
 * and receives the final one. dt > 0, nsteps >= 0.
 */
int dg_step_lsrk(dg_ctx* ctx, void* U, double dt, int32_t nsteps, uintptr_t stream);

/*
 * Low-storage Runge-Kutta scheme that dg_step_lsrk (and dg_solve_host with
 * method 0) runs on this context (Sec. 2.2, Table crit-Cr):
 *   DG_LSRK_CK54  the 2N-storage five-stage fourth-order scheme above
 *                 (the default);
 *   DG_LSRK45     the paper's LSRK4(5), the two-register RK4(3)5[2R+]C of
 *                 Kennedy, Carpenter & Lewis (five stages, order four);
 *   DG_LSRK59     the paper's LSRK5(9), RK5(4)9[2R+]S (nine stages, order
 *                 five).
 * A two-register stage i evaluates R at its input Y_i and, fused into the
 * operator's epilogue, writes Y_{i+1} = S_i + dt A_i R(Y_i) and
 * S_{i+1} = S_i + dt B_i R(Y_i), with Y_1 = S_1 = u_n and u_{n+1} = S_{s+1}:
 * four state passes per stage (three in the first and last). Both storage
 * bases and both precisions. DG_EINVAL for another value; DG_EUNSUPPORTED
 * for a two-register scheme on a 2D context. Batches and partitioned solves
 * step the default scheme only (their LSRK calls return DG_EUNSUPPORTED on
 * contexts set otherwise).
 */
#define DG_LSRK_CK54 0
#define DG_LSRK45 1
#define DG_LSRK59 2
int dg_set_lsrk_scheme(dg_ctx* ctx, int32_t scheme);
/* The context's scheme, or DG_EINVAL for NULL. */
int dg_get_lsrk_scheme(const dg_ctx* ctx);

/*
 * nsteps of ADER (Sec. 2.3, Eq. (6)): Ubar = Taylor-Cauchy-Kowalevski
 * predictor with the element-local basis change GL -> G (Sec. 3.2,
 * Algorithm 2) and degree reduction every reduce_every-th derivative
 * (Sec. 3.3, Algorithm 3; 2 = the paper's choice, 0 = none, 1 and 3 = the
 * other variants of Fig. reduc-comp), then U <- U - M^-1 K Ubar. Sum over
 * j = 0..k+1. Other values of reduce_every return DG_EUNSUPPORTED.
 * Reductions by 1 or 3 visit Gauss sets that the set-up does not store by
 * default (it stores n, n-2, ...): on a mesh that is curved or has
 * variable coefficients, the first such call synchronises the stream,
 * allocates the predictor data of every set n, n-1, ..., 2 and recomputes
 * the geometry (an extra 11 sum_m m^3 values per element at most).
 */
int dg_step_ader(dg_ctx* ctx, void* U, double dt, int32_t nsteps,
                 int32_t reduce_every, uintptr_t stream);

/*
 * nsteps of HDG-ADER (Sec. 2.4, Eq. hdg-ader): every step first evaluates the
 * DG derivative W = -M^-1 K U (one more operator application), which takes
 * the place of the predictor's first Taylor term -S U; then
 * U <- U - M^-1 K Ubar as in dg_step_ader. The HDG flux with tau = 1/(rho c)
 * is the upwind flux of this build (flux_alpha = 1) where rho c is continuous.
 * The superconvergent postprocessing the paper refers to is not part of it.
 * Arguments, errors and the storage basis as for dg_step_ader.
 */
int dg_step_hdg_ader(dg_ctx* ctx, void* U, double dt, int32_t nsteps,
                     int32_t reduce_every, uintptr_t stream);

/*
 * Representation of the state inside dg_step_lsrk and dg_step_ader (the
 * state passed in and out is always GL nodal values):
 *  DG_BASIS_GL  the paper's scheme: GL storage, so that a face needs only the
 *               neighbour's (k+1)^2 face nodes, and an on-the-fly change to
 *               the collocated Gauss basis inside each element (Sec. 3.1-3.2).
 *  DG_BASIS_G   values at the Gauss points during the steps: the steppers
 *               change basis once on entry and once on exit; the operator
 *               then needs no basis change and a diagonal mass matrix, and a
 *               face reads the neighbour's line of (k+1) values through each
 *               face point. Same discrete scheme; fewer arithmetic operations
 *               and more face data, the trade-off the paper measures
 *               (Sec. 3.1), which favours G where arithmetic is scarce (FP64
 *               on GB300).
 * Default DG_BASIS_GL.
 */
#define DG_BASIS_GL 0
#define DG_BASIS_G 1
int dg_set_basis(dg_ctx* ctx, int basis);
int dg_get_basis(const dg_ctx* ctx);

/*
 * Predictor kernel for Gauss-point states (DG_BASIS_G steppers, dg_tck is
 * unaffected).  Both compute the Taylor sum of Sec. 2.3 Eq. (6) with the
 * degree reduction of Sec. 3.3, to rounding:
 *  DG_PRED_LINES    every derivative, projection and prolongation as
 *                   contractions of element tiles in shared memory, lines
 *                   spread over the whole block;
 *  DG_PRED_COLUMNS  each thread keeps a z-column of the current Taylor term
 *                   and of the n-point sum in registers; x and y lines pass
 *                   through shared memory once per derivative;
 *  DG_PRED_INTERLEAVED
 *                   the column form with the block's elements interleaved in
 *                   shared memory and the state staged by bulk copies, for
 *                   FP32 meshes of affine elements with constant
 *                   coefficients, reduce_every 0 or 2 and no HDG
 *                   derivative (elsewhere the column form runs): fewer
 *                   shared-memory bank conflicts and idle lanes, and each
 *                   reduced Taylor term formed on the smaller Gauss set with
 *                   the projected derivative (Sec. 3.3); the column form's
 *                   results up to FP32 rounding;
 *  DG_PRED_AUTO     the interleaved form where it applies, else the column
 *                   form, in FP32; the line form in FP64 (default; the FP64
 *                   pipe is the bound there, and the line form keeps whole
 *                   warps busy at the reduced Gauss sets).
 *  DG_PRED_GL_PROJECTION
 *                   the predictor without the basis change (Sec. 3.2,
 *                   Alg. 1), for GL states (DG_BASIS_GL steppers and dg_tck)
 *                   with reduce_every 0: each derivative is evaluated at the
 *                   Gauss points, integrated against the GL functions and
 *                   projected with the inverse GL mass matrix.  Equal to the
 *                   other forms in exact arithmetic, several times their
 *                   work; it exists to measure what Secs. 3.2-3.3 save.
 *                   Other states or reductions, and HDG-ADER, return
 *                   DG_EUNSUPPORTED when a predictor runs.
 * Takes effect on 3D contexts stepped on their own.  Batches (and so the
 * server) choose for themselves: the column form for FP32 Gauss-point
 * states, the line form otherwise; each batched solve then matches the same
 * solve stepped alone with DG_PRED_AUTO bit for bit, except an FP32 solve
 * on affine elements with constant coefficients, which runs the interleaved
 * form alone and agrees to FP32 rounding.  Errors: DG_EINVAL,
 * DG_EUNSUPPORTED (DG_PRED_GL_PROJECTION on a 2D context).
 */
#define DG_PRED_AUTO 0
#define DG_PRED_LINES 1
#define DG_PRED_COLUMNS 2
#define DG_PRED_GL_PROJECTION 3
#define DG_PRED_INTERLEAVED 4
int dg_set_predictor_kernel(dg_ctx* ctx, int kind);
int dg_get_predictor_kernel(const dg_ctx* ctx);

/*
 * 1 if every element is an affine image of the reference cube and the
 * coefficients are constant within each element (checked at set-up and at
 * dg_set_coefficients), else 0. Such meshes get compact per-element data
 * (metric, mass and face constants times Gauss weights) in the Gauss-basis
 * operator and in the predictor: same scheme, much less data to read.
 */
int dg_is_affine(const dg_ctx* ctx);

/* In-place change of basis of a device state: GL -> G (to_g != 0) or G -> GL. */
int dg_change_basis(dg_ctx* ctx, void* U, int to_g, uintptr_t stream);

/*
 * The predictor alone: Ubar (device, GL basis) = sum_j dt^{j+1}/(j+1)! T_j of
 * Eq. (6) for the state U. U and Ubar must not overlap. reduce_every as for
 * dg_step_ader (0, 1, 2 or 3).
 */
int dg_tck(dg_ctx* ctx, const void* U, void* Ubar, double dt, int32_t reduce_every,
           uintptr_t stream);

/*
 * Discrete energy 1/2 U^T M U = 1/2 (rho |v|^2 + p^2/(rho c^2)) integrated by
 * the Gauss rule, accumulated in double with a fixed summation order
 * (bitwise reproducible). *out is a host double; the call synchronises the
 * stream.
 */
int dg_energy(dg_ctx* ctx, const void* U, double* out, uintptr_t stream);

/*
 * dg_energy without allocation.  The paper has no counterpart to this call;
 * it exists for callers that must not allocate device memory once they are
 * running: a serving process that has promised its whole HBM budget to
 * admitted solves, code whose memory use is fixed and checked up front, or a
 * latency-critical loop where cudaMalloc/cudaFree would synchronise the
 * device and stall other streams.
 *
 * Computes the same value as dg_energy for the device state U and writes it
 * to *out, a caller-owned device double, on the given stream (no host
 * synchronisation; read *out after the stream's work completes).  The
 * partial sums go to one fixed device array of 16384 doubles (128 KB) that
 * every GPU loading the library holds until the process exits; meshes that
 * need more partial sums than that (more than 16384 blocks of the energy
 * kernel, e.g. more than 49152 elements at k = 5 in FP64) are rejected with
 * DG_EINVAL and a message naming the limit.  The call makes no cudaMalloc or
 * cudaFree and, when it succeeds, no host allocation.
 *
 * The first call on a device resolves the device address of that array with
 * the device current (this may load the library's device code), so make that
 * first call before capturing any stream.  All calls on a device share the
 * array: calls whose GPU work overlaps (different streams, no ordering)
 * race on it and give wrong results; calls on one stream are safe.  Each
 * call writes every slot it reads, so nothing from an earlier call leaks in.
 */
int dg_energy_noalloc(dg_ctx* ctx, const void* U, double* out, uintptr_t stream);

/*
 * Sums of squares over all entries, accumulated in double in a fixed order:
 * *out_aa = sum A^2 and, when B is not NULL, *out_dd = sum (A - B)^2.
 * A, B are device states of this context. Synchronises the stream.
 */
int dg_norms(dg_ctx* ctx, const void* A, const void* B, double* out_aa,
             double* out_dd, uintptr_t stream);

/*
 * End-to-end solve through host memory: copy U_host (host, [E][4][(k+1)^3]
 * in the context precision) into a context-owned device state, run nsteps of
 * method (0 = LSRK, 1 = ADER), copy the result back to U_out_host, and
 * synchronise. When the context steps with Gauss-point states (DG_BASIS_G,
 * 3D) and both host buffers are pinned (page-locked, mapped) or managed
 * memory, 16-byte aligned, the transfers are fused with the two changes of
 * basis: one kernel reads U_host through the device's mapping and writes the
 * Gauss-point values, another writes the GL result straight into
 * U_out_host. Pageable buffers take plain copies instead (same results).
 */
int dg_solve_host(dg_ctx* ctx, int method, const void* U_host, void* U_out_host,
                  double dt, int32_t nsteps, int32_t reduce_every, uintptr_t stream);

/*
 * Checkpoint and restart of a solve.  The paper's steppers are one-step
 * methods (Sec. 2.2-2.3: the LSRK stages and the ADER step need only U_n),
 * so U between two step calls is the whole state of a solve: a restart
 * from it gives, bit for bit, what the same step calls give without the
 * checkpoint.  (With DG_BASIS_G a call changes basis on entry and exit, so
 * two calls of m steps and one call of 2m steps agree to rounding only.)
 *
 * dg_get_state copies the device state U (this context's precision and
 * layout, [E][fields][npts] in the Gauss-Lobatto basis) into the caller's
 * host array host_out of E*fields*npts doubles (fields = 4 and npts =
 * (k+1)^3 in 3D; 3 and (k+1)^2 in 2D).  dg_set_state copies such a host
 * array into the device state U, rounding to nearest when the context is
 * FP32.  FP32 -> FP64 -> FP32 is exact, so a checkpoint of either precision
 * restores bit for bit.  For an FP32 context each call takes a temporary
 * device buffer of 8 bytes per entry from the stream-ordered allocator and
 * returns it before it returns (DG_ENOMEM if that fails).  Host arrays may
 * be pageable; both calls synchronise the stream.  A partitioned context
 * copies its whole local state, ghost slots included.
 */
int dg_get_state(dg_ctx* ctx, const void* U, double* host_out, uintptr_t stream);
int dg_set_state(dg_ctx* ctx, const double* host_in, void* U, uintptr_t stream);

/*
 * Per-kernel timing. While enabled, every kernel launch of the context is
 * bracketed by two CUDA events recorded on the launching stream.
 * dg_profile_read synchronises on those events and returns, per kind, the
 * summed device time in ms and the number of launches since the last reset
 * (arrays of DG_NKINDS entries); reset != 0 starts a new interval.
 */
#define DG_KIND_OPERATOR 0 /* R = -M^-1 K U alone */
#define DG_KIND_LSRK 1     /* operator fused with one LSRK stage update */
#define DG_KIND_ADER 2     /* operator fused with the ADER update */
#define DG_KIND_TCK 3      /* Taylor-Cauchy-Kowalevski predictor */
#define DG_KIND_OTHER 4    /* set-up, energy, norms */
#define DG_NKINDS 5
int dg_profile_enable(dg_ctx* ctx, int enable);
int dg_profile_read(dg_ctx* ctx, double* ms, int64_t* launches, int reset);

/*
 * Tiling: elements per thread block of the operator kernels (epb_op) and of
 * the predictor (epb_tck); each element gets (k+1)^2 threads. Values <= 0
 * leave a setting unchanged; impossible values (over 1024 threads or the
 * shared-memory budget) give DG_EINVAL. Results do not depend on tiling.
 */
int dg_set_tiling(dg_ctx* ctx, int32_t epb_op, int32_t epb_tck);
int dg_get_tiling(const dg_ctx* ctx, int32_t* epb_op, int32_t* epb_tck);

/*
 * Measure one kernel kind (DG_KIND_LSRK, DG_KIND_ADER or DG_KIND_TCK), in the
 * variant the steppers use for the context's basis, on this context's mesh
 * for each candidate elements-per-block value: ms_out[c] =
 * device ms per launch (average of reps), -1 for impossible candidates. The
 * fastest candidate is left set. Uses context scratch; synchronises.
 */
int dg_tune(dg_ctx* ctx, int kind, const int32_t* cand, int32_t ncand, int32_t reps,
            double* ms_out, uintptr_t stream);

/*
 * Batched form: n independent solves (different meshes, degrees, time steps;
 * one precision, one device) advanced together. For each degree present,
 * each phase of a step (the LSRK stages; the ADER predictor and update) is
 * one persistent launch over work items (runs of consecutive elements of one
 * solve; largest solves first, each in element order) taken dynamically by
 * the blocks; the degrees run as
 * concurrent branches forked from and joined to the caller's stream. Chunks
 * of 8 steps are captured once as a CUDA graph and replayed. Every element runs the same arithmetic as in the
 * single-solve calls, so each solve's result is bitwise identical to running
 * it alone. U[i] are the solves' device states (updated in place), dt[i]
 * their time steps; contexts and states must outlive the batch.
 */
typedef struct dg_batch dg_batch;
int dg_batch_create(dg_ctx* const* ctxs, void* const* U, const double* dt, int32_t n,
                    uintptr_t stream, dg_batch** out);
/* reduce_every 0 or 2 here; 1 and 3 return DG_EUNSUPPORTED (use dg_step_ader per solve). */
int dg_batch_step_ader(dg_batch* b, int32_t nsteps, int32_t reduce_every, uintptr_t stream);
int dg_batch_step_lsrk(dg_batch* b, int32_t nsteps, uintptr_t stream);
/*
 * State basis of a batch's steps (DG_BASIS_GL default, or DG_BASIS_G as for
 * dg_set_basis). With DG_BASIS_G and convert_each_call != 0 every step call
 * changes the states to the Gauss basis on entry and back on exit; with 0 the
 * states stay in whatever basis the caller keeps them in, and the caller
 * changes basis with dg_batch_convert or dg_change_basis (a solve's result
 * then does not depend on how its steps are split into calls).
 */
int dg_batch_set_basis(dg_batch* b, int basis, int convert_each_call);
int dg_batch_convert(dg_batch* b, int to_g, uintptr_t stream);
int dg_batch_info(const dg_batch* b, int32_t* n_inst, int32_t* n_items, int32_t* block,
                  int32_t* grid, uint64_t* launches);
const char* dg_batch_last_error(const dg_batch* b);
void dg_batch_destroy(dg_batch* b);

/*
 * Partitioned solve (the data-parallel split of one solve, Sec. 4.1, 4.8: the
 * operator needs the neighbours' data across a face, the predictor none).
 * A part is a context set up on its owned elements followed by ghost
 * elements: copies of the neighbours of owned elements that other parts own.
 * Ghosts keep their faces towards elements present in the part and have
 * walls elsewhere; they are never stepped.
 *
 * dg_set_owned: only the first n_owned elements of ctx are stepped (default
 * all); operator, predictor, basis changes, energy and norms then cover those
 * elements alone. 1 <= n_owned <= element count, else DG_EINVAL.
 *
 * dg_part_create: ctxs[P], U[P] (device states of the parts, [E_i][4][n^3],
 * 16-byte aligned, caller-owned, must outlive the object), n_ghost[P] with
 * n_owned_i + n_ghost[i] == E_i. ghost_src_part / ghost_src_elem list, part
 * after part and in each part's ghost order, the owning part (!= the ghost's
 * own part) and its owned element index of every ghost. Parts must share
 * degree, precision, device and storage basis (dg_set_basis). Copies the map
 * to the device (a small allocation), so create once and step many times.
 * Errors: DG_EINVAL (message in dg_last_error(NULL)), DG_ENOMEM.
 *
 * dg_part_step_lsrk / dg_part_step_ader: as dg_step_lsrk / dg_step_ader for
 * the whole mesh. Before every operator application the ghost tiles of its
 * input (the stage input for LSRK, the predictor for ADER) are copied from
 * their owners by one gather kernel on the stream: five exchanges per LSRK
 * step, one per ADER step. Every owned element then computes exactly what it
 * computes in the unpartitioned solve, so the owned states are bitwise equal
 * to those of one context on the whole mesh that runs the same kernels (the
 * same storage basis, and every part affine or not as the whole mesh is).
 * dg_part_exchange copies the ghosts of the states U themselves.
 */
int dg_set_owned(dg_ctx* ctx, int32_t n_owned);
typedef struct dg_part dg_part;
int dg_part_create(dg_ctx* const* ctxs, void* const* U, int32_t P, const int32_t* n_ghost,
                   const int32_t* ghost_src_part, const int32_t* ghost_src_elem, dg_part** out);
int dg_part_step_lsrk(dg_part* t, double dt, int32_t nsteps, uintptr_t stream);
int dg_part_step_ader(dg_part* t, double dt, int32_t nsteps, int32_t reduce_every, uintptr_t stream);
/* HDG-ADER on the parts: two exchanges per step (the state, then the predictor). */
int dg_part_step_hdg_ader(dg_part* t, double dt, int32_t nsteps, int32_t reduce_every, uintptr_t stream);
int dg_part_exchange(dg_part* t, uintptr_t stream);
int dg_part_info(const dg_part* t, int32_t* n_parts, int32_t* n_ghost_total, uint64_t* exchanges);
const char* dg_part_last_error(const dg_part* t);
void dg_part_destroy(dg_part* t);

/*
 * Served form: continuous batching of solves on one GPU. An admission thread
 * takes queued requests in arrival order while they fit the HBM budget (a
 * request that does not fit lets later, smaller ones in) and sets them up on
 * the device on its own stream while the GPU keeps stepping; a stepping
 * thread keeps each admitted solve's geometry and state device-resident and
 * advances all admitted solves together (dg_batch) in rounds of at most
 * chunk_steps steps, ending a round when a solve finishes. Finished states are copied to the caller's
 * buffer and their memory released; requests that arrived meanwhile join at
 * the next round. Each result is bitwise identical to solving it alone
 * with the predictor form batches run (dg_set_predictor_kernel: for an
 * FP32 solve on affine elements with constant coefficients that is the
 * column form, where DG_PRED_AUTO alone runs the interleaved form and
 * agrees to FP32 rounding).
 */
typedef struct dg_server dg_server;
typedef struct {
  int32_t device;      /* CUDA device index */
  int32_t prec;        /* DG_FP32 or DG_FP64 */
  int32_t max_active;  /* most solves admitted at once; 0 = only the budget limits */
  int32_t chunk_steps; /* steps per round at most; 0 = 16 */
  double max_active_dof; /* admit only while the admitted solves hold fewer
                            DoFs than this (0 = no limit): enough to fill the
                            GPU, so that early requests finish early */
} dg_server_opts;
typedef struct {
  dg_mesh_desc mesh;   /* as for dg_mesh_setup; copied at submit */
  int32_t k;
  double flux_alpha;
  const double* rho;   /* [E][(k+1)^3], copied at submit */
  const double* c;     /* [E][(k+1)^3], copied at submit */
  const void* U0;      /* host [E][4][(k+1)^3] in the server precision, copied */
  void* U_out;         /* host buffer for the final state (server precision);
                          caller-owned, must stay valid until dg_poll gives
                          DG_OK for this request */
  double dt;
  int32_t nsteps;
  int32_t method;      /* 0 = LSRK(5,4), 1 = ADER */
  int32_t reduce_every; /* 0 or 2 (the server steps requests in batches) */
} dg_request;
typedef struct {
  double t_submit, t_admit, t_done; /* seconds, one monotonic clock */
  int32_t status;                   /* DG_OK or the error of this solve */
} dg_result;
typedef struct {
  int32_t queued, active, peak_active;
  uint64_t completed, rounds, batches_built;
  size_t hbm_used, hbm_peak;  /* budget accounting, bytes */
  double dof_steps;           /* DoF-steps advanced so far */
  double busy_s;              /* time spent in stepping rounds */
} dg_server_stats_t;

/* Device bytes the server reserves from its budget for one admitted solve
 * (geometry, coefficients, state and all scratch); 0 for invalid sizes. */
size_t dg_request_bytes(int32_t n_elem, int32_t k, int32_t geom_degree, int32_t prec);

/* Start a server on opts->device with an HBM budget in bytes. */
int dg_server_create(size_t hbm_budget, const dg_server_opts* opts, dg_server** out);
/* Queue a request (never blocks on the GPU); DG_ENOMEM if it can never fit
 * the budget, DG_EINVAL for a malformed request. */
int dg_submit(dg_server* s, const dg_request* r, uint64_t* ticket);
/* DG_EAGAIN until the request is finished (waiting up to timeout_ms), then
 * DG_OK with *out filled; a ticket can be polled to completion once. */
int dg_poll(dg_server* s, uint64_t ticket, dg_result* out, int32_t timeout_ms);
int dg_server_stats(dg_server* s, dg_server_stats_t* out);
/* Stop the scheduling thread and free everything; unfinished requests are
 * dropped. */
void dg_server_destroy(dg_server* s);

/*
 * Device status: DG_ETIMEOUT if, since the last check, a kernel of this
 * context gave up a bounded wait (its shared-memory staging did not complete
 * in time; that block's results were discarded), else DG_OK. Synchronises
 * the stream and clears the status. dg_solve_host checks it itself.
 */
int dg_check_device(dg_ctx* ctx, uintptr_t stream);

/*
 * Testing only (no counterpart in the paper): with on != 0, the first
 * bounded wait of the kernels that stage their inputs by bulk copy (the FP32
 * Gauss-basis operators) gives up at once instead of after its poll limit.
 * The kernel then runs its give-up path as it would after a real stall: it
 * sets the device status, waits (bounded) for its own copies to land, and
 * returns without writing results, so the next dg_check_device reports
 * DG_ETIMEOUT. Nothing hangs and the context stays usable; on = 0 restores
 * normal operation. Other kernels are unaffected. DG_EINVAL for a NULL ctx.
 */
int dg_test_expire_waits(dg_ctx* ctx, int32_t on);

/*
 * Measurement helper (no counterpart in the paper): the FMA pipe's peak in
 * TFLOP/s on the current device, DG_FP64 or DG_FP32, from one timed launch
 * of independent FMA chains (8 per thread, iters FMAs each, 8 blocks of 256
 * threads per SM) after one untimed launch, on the given stream. These are
 * the measured denominators of the ALU rooflines. Allocates nothing (a
 * static device word keeps the chains live). DG_EINVAL for bad arguments,
 * DG_ECUDA if a CUDA call fails.
 */
int dg_probe_fma_peak(int32_t prec, int32_t iters, double* tflops, uintptr_t stream);

/* Sizes: number of elements, degree, precision, bytes of one state. */
int dg_info(const dg_ctx* ctx, int32_t* n_elem, int32_t* k, int32_t* prec,
            size_t* state_bytes);

/* Device bytes owned by the context (geometry, coefficients, scratch). */
size_t dg_device_bytes(const dg_ctx* ctx);

/* Kernel launches issued by this context since it was created. */
uint64_t dg_launch_count(const dg_ctx* ctx);

/* Free everything owned by the context. NULL-safe. */
void dg_destroy(dg_ctx* ctx);

/* Static string for a status code. */
const char* dg_strerror(int status);

/* Last error message of the context ("" if none); NULL ctx gives the
 * message of the last failed dg_mesh_setup in this thread. */
const char* dg_last_error(const dg_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* DG_H */
