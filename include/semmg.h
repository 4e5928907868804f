/*
 * semmg -- p-multigrid for the statically condensed spectral-element Helmholtz
 * problem on one GPU (sm_103a).  C ABI.
 *
 * Method: Huismann, Stiller, Froehlich, "Scaling to the stars -- a linearly
 * scaling elliptic solver for p-multigrid", arXiv:1808.03595.
 *
 * Problem (Sec. 2.1, eq. helmholtz_equation): lambda u - Laplace u = f on a box
 * meshed by a tensor product of cuboidal elements (per-axis widths h_d[a]),
 * GLL nodal basis of degree p.  Each face of the box is Dirichlet (homogeneous,
 * or with data g through semmg_solve_dirichlet / semmg_pack_dirichlet),
 * homogeneous Neumann, or periodic (both faces of an axis), Sec. 3.3; see
 * semmg_mesh.bc.  The element operator is eq. helmholtzop with coefficients
 * d_e = h1 h2 h3 / 8 (lambda, 4/h1^2, 4/h2^2, 4/h3^2), the rightmost Kronecker
 * factor acting along x1.
 *
 * ------------------------------------------------------------------ layouts
 * Nodal arrays: the global GLL grid of a level, N_d = n_d p + 1 points per
 * axis, FP64, C order u[g3][g2][g1] (x1 fastest), boundary planes included
 * (on a periodic axis the last plane is the image of the first).
 *
 * Condensed ("hat") vectors: values on the element skeleton (element-boundary
 * nodes, Sec. 2.2), one slot per unique node, grouped by entity, with m = p-1,
 * nv_d = n_d + 1 vertex planes per axis.  Every vertex plane has slots, also
 * where it holds no unknowns:
 *   - on a Dirichlet face the slots are not unknowns.  Every output of the
 *     operator, residual, smoother and transfers is 0 there; an input vector
 *     may carry Dirichlet data there (semmg_pack_dirichlet), which the
 *     operator, residual and recovery read as prescribed boundary values;
 *   - on a Neumann face the slots are unknowns like interior ones;
 *   - the last vertex plane of a periodic axis repeats plane 0: its slots are
 *     never read and outputs leave them 0.
 * Group order and index formulas (c = vertex-plane index,
 * a = element index, i = 0..m-1 interior node index, the last index fastest):
 *   F1 faces normal to x1 [a3][a2][c1][i3][i2]   n3 n2 nv1 m^2
 *   F2 faces normal to x2 [a3][c2][a1][i3][i1]   n3 nv2 n1 m^2
 *   F3 faces normal to x3 [c3][a2][a1][i2][i1]   nv3 n2 n1 m^2
 *   E1 edges along x1     [c3][c2][a1][i1]       nv3 nv2 n1 m
 *   E2 edges along x2     [c3][a2][c1][i2]       nv3 n2 nv1 m
 *   E3 edges along x3     [a3][c2][c1][i3]       n3 nv2 nv1 m
 *   V  vertices           [c3][c2][c1]           nv3 nv2 nv1
 * Levels are numbered 0 (coarsest, degree p0) .. L (finest, degree p); the
 * degrees are p_l = p0 2^l for l < L and p_L = p (Sec. 4.1).
 *
 * ------------------------------------------------------------------ ownership
 * Every vector argument is a DEVICE pointer owned by the caller, except in
 * semmg_solve_host, whose f/u are HOST pointers.  The library allocates its
 * tables and work buffers in semmg_setup (cudaMalloc) and frees them in
 * semmg_destroy.  Every call is ordered on `stream` (a cudaStream_t, NULL =
 * legacy default stream) and asynchronous unless stated otherwise.  A context
 * is not thread-safe: calls on one context must not overlap in time on the
 * host, and calls on one context enqueued on different streams race on its
 * work buffers.
 *
 * ------------------------------------------------------------------ errors
 * Every function returns SEMMG_OK (0) or a negative SEMMG_ERR_* code and never
 * aborts the process.  semmg_last_error() gives a message for the last failure
 * on a context (including the CUDA error string for SEMMG_ERR_CUDA).
 */
#ifndef SEMMG_H
#define SEMMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct semmg_ctx semmg_ctx;

enum {
  SEMMG_OK = 0,
  SEMMG_ERR_INVALID_ARG = -1,   /* null pointer, bad size, level out of range */
  SEMMG_ERR_UNSUPPORTED = -2,   /* p < 1, p > SEMMG_MAX_DEGREE, p0 > p, ... */
  SEMMG_ERR_CUDA = -3,          /* a CUDA runtime call failed */
  SEMMG_ERR_NOT_CONVERGED = -4, /* max_iter cycles without reaching rtol; info filled */
  SEMMG_ERR_NONFINITE = -5,     /* NaN or Inf in a residual norm */
  SEMMG_ERR_TIMEOUT = -6,       /* a bounded device wait ran out (tensor-core smoother, semmg_set_guards) */
  SEMMG_ERR_NOMEM = -7,         /* device or host allocation failed */
  SEMMG_ERR_DIVERGED = -8       /* the residual norm grew above 1e3 ||r_0|| (semmg_set_guards): stopped early;
                                   info filled */
};

#define SEMMG_MAX_DEGREE 48

/* precision of the V-cycle; the outer iteration (its residual, norms and
 * update) and the coarse solve are always FP64, and so are condensation and
 * recovery except in the solves of the float-float forms.
 *   SEMMG_FP64        everything FP64;
 *   SEMMG_MIXED       FP32 vectors, smoother and transfers in the V-cycle; its
 *                     level residuals F - Hhat u in FP64 arithmetic on the FP32
 *                     values (rounded once to FP32);
 *   SEMMG_MIXED_FP32  the whole V-cycle in FP32, level residuals included;
 *   SEMMG_MIXED_TC    as SEMMG_MIXED, with the star smoother's 1D transforms on
 *                     tensor cores (tcgen05, TF32 operands, FP32 accumulation)
 *                     on the levels with 16 <= p <= 48; other levels as SEMMG_MIXED;
 *   SEMMG_MIXED_FP32_TC  as SEMMG_MIXED_FP32, with the tensor-core smoother of
 *                     SEMMG_MIXED_TC on the levels it covers;
 *   SEMMG_MIXED_BF16  as SEMMG_MIXED_TC with BF16 operands (8-bit significand,
 *                     FP32 accumulation) in the tensor-core transforms;
 *   SEMMG_MIXED_FF    as SEMMG_MIXED, with the level residuals of the levels
 *                     with p >= 12 (the face-parallel form of the operator) in
 *                     float-float arithmetic: every value an unevaluated sum of
 *                     two FP32 numbers (about 48 significant bits), run on the
 *                     FP32 pipes; levels with p < 12 as SEMMG_MIXED.  When the
 *                     finest level has p >= 12, semmg_solve (and a batch) also
 *                     condenses the right-hand side and recovers the interiors
 *                     in float-float (relative rounding about 1e-14, four
 *                     orders below the 1e-10 target); semmg_condense_rhs and
 *                     semmg_recover stay FP64;
 *   SEMMG_MIXED_FF_TC as SEMMG_MIXED_FF, with the tensor-core smoother of
 *                     SEMMG_MIXED_TC. */
enum {
  SEMMG_FP64 = 0,
  SEMMG_MIXED = 1,
  SEMMG_MIXED_FP32 = 2,
  SEMMG_MIXED_TC = 3,
  SEMMG_MIXED_FP32_TC = 4,
  SEMMG_MIXED_BF16 = 5,
  SEMMG_MIXED_FF = 6,
  SEMMG_MIXED_FF_TC = 7
};
/* outer iteration of semmg_solve and of the batched form */
enum { SEMMG_SOLVER_MG = 0, SEMMG_SOLVER_KMG = 1 };
/* Schwarz smoother of the V-cycle levels */
enum {
  SEMMG_SMOOTHER_STAR = 0,         /* vertex stars, Algorithm 2 around Algorithm 1 (Sec. 3.2), default */
  SEMMG_SMOOTHER_ELEMENT = 1,      /* element-centred 3x3x3-element blocks with full overlap (Sec. 3.4),
                                      weights one on the element's own nodes, zero on the other elements',
                                      one half on faces shared with a neighbour block */
  SEMMG_SMOOTHER_ELEMENT_MULT = 2  /* the same blocks, inverse-multiplicity weights (Sec. 2.3) */
};  /* the element-centred smoothers need n[d] >= 3 on periodic axes */
/* element type of a vector argument of smooth / restrict / prolong_add */
enum { SEMMG_F64 = 0, SEMMG_F32 = 1 };

/* boundary condition of a face of the domain (Sec. 3.3) */
enum { SEMMG_BC_DIRICHLET = 0, SEMMG_BC_NEUMANN = 1, SEMMG_BC_PERIODIC = 2 };

typedef struct {
  int n[3];              /* elements per axis, each >= 1 */
  const double* h[3];    /* HOST arrays: n[d] element widths along axis d, > 0 */
  int bc[6];             /* faces -x1, +x1, -x2, +x2, -x3, +x3: SEMMG_BC_DIRICHLET (0, homogeneous,
                            the value of a zero-initialised struct), SEMMG_BC_NEUMANN (homogeneous:
                            the face's nodes are unknowns, the ghost element beyond it is decoupled)
                            or SEMMG_BC_PERIODIC (both faces of an axis, n[d] >= 2: the ghost element
                            is the element at the other end; nodal arrays keep n[d] p + 1 planes along
                            d, the last one the image of the first).  Without a Dirichlet face
                            lambda must be > 0. */
} semmg_mesh;

typedef struct {
  int p0;          /* coarse degree, 1 <= p0 <= p (default 2, Sec. 4.1) */
  int nu_pre;      /* pre-smoothing steps per level (default 1, Algorithm 3) */
  int nu_post;     /* post-smoothing steps per level (default 1) */
  int precision;   /* SEMMG_FP64 (default), SEMMG_MIXED, SEMMG_MIXED_FP32, SEMMG_MIXED_TC, SEMMG_MIXED_FP32_TC,
                      SEMMG_MIXED_BF16, SEMMG_MIXED_FF or SEMMG_MIXED_FF_TC */
  int max_iter;    /* iteration cap of semmg_solve (default 50; 0: condensation and recovery from u_hat = 0 only) */
  int solver;      /* SEMMG_SOLVER_MG (Algorithm 4, default) or SEMMG_SOLVER_KMG (Algorithm 5) */
  int nu_vary;     /* 0 (default): nu_pre / nu_post steps on every level; 1: nu_pre 2^(L-l) and
                      nu_post 2^(L-l) steps on level l (Sec. 4.1, "kvMG" with SEMMG_SOLVER_KMG) */
  int smoother;    /* SEMMG_SMOOTHER_STAR (default), SEMMG_SMOOTHER_ELEMENT or SEMMG_SMOOTHER_ELEMENT_MULT */
} semmg_opts;

typedef struct {
  int iters;          /* V-cycles performed (n_10 when rtol = 1e-10) */
  double res0;        /* ||r_0||_2 over the condensed unknowns */
  double res_final;   /* ||r_iters||_2 */
  double rho;         /* (res_final / res0)^(1/iters), Sec. 5.2 */
  int status;         /* return code of the solve */
} semmg_info;

/* Fill *opts with the defaults listed above. */
void semmg_default_opts(semmg_opts* opts);

/* Build the level hierarchy of Sec. 4.1 for the mesh, degree p and lambda >= 0:
 * 1D GLL tables, element interior eigenpairs, per-vertex-line star eigen-tables
 * with identity padding at the Dirichlet boundary (Sec. 3.2-3.3), smoother
 * weights (degree 7, Sec. 3.2), interpolation matrices and the coarse
 * fast-diagonalisation tables; uploads them and allocates work buffers.
 * opts may be NULL (defaults).  Synchronises the device once at the end.
 * On success *out owns everything; release it with semmg_destroy. */
int semmg_setup(const semmg_mesh* mesh, int p, double lambda, const semmg_opts* opts,
                void* stream, semmg_ctx** out);

/* Free all device and host memory of ctx (NULL is ignored).  Synchronises. */
void semmg_destroy(semmg_ctx* ctx);

/* Number of levels L+1 and the degree of a level. */
int semmg_num_levels(const semmg_ctx* ctx, int* nlevels);
int semmg_level_degree(const semmg_ctx* ctx, int level, int* p);

/* Length of a condensed vector (skeleton slots, boundary ones included) and of
 * a nodal array, at a level. */
int semmg_condensed_size(const semmg_ctx* ctx, int level, int64_t* n);
int semmg_nodal_size(const semmg_ctx* ctx, int level, int64_t* n);

/* Condensed <-> nodal copies at a level (FP64).  pack reads the skeleton nodes
 * of u_nodal (zero written on the Dirichlet boundary); unpack writes the
 * skeleton nodes of u_nodal and leaves element-interior nodes untouched. */
int semmg_pack(semmg_ctx* ctx, int level, const double* u_nodal, double* u_hat, void* stream);
int semmg_unpack(semmg_ctx* ctx, int level, const double* u_hat, double* u_nodal, void* stream);

/* u_hat = E g: the values of the nodal array g_nodal at the nodes on Dirichlet
 * faces copied into their (boundary) skeleton slots, zero in every other slot.
 * A condensed vector whose boundary slots hold Dirichlet data is read by
 * semmg_apply_condensed, semmg_residual and semmg_recover as the prescribed
 * boundary values (the lifting of inhomogeneous Dirichlet data, used by the
 * paper's test problem of Sec. 5.2); their outputs stay zero in those slots. */
int semmg_pack_dirichlet(semmg_ctx* ctx, int level, const double* g_nodal, double* u_hat, void* stream);

/* y_hat = Hhat u_hat, Hhat = H_BB - H_BI H_II^{-1} H_IB the condensed operator
 * (Sec. 2.2) applied matrix-free in O(p^3) per element, FP64.  y_hat must not
 * alias u_hat. */
int semmg_apply_condensed(semmg_ctx* ctx, int level, const double* u_hat, double* y_hat, void* stream);

/* r_hat = f_hat - Hhat u_hat (Sec. 2.3, residual), FP64.  r_hat may alias f_hat. */
int semmg_residual(semmg_ctx* ctx, int level, const double* f_hat, const double* u_hat,
                   double* r_hat, void* stream);

/* r_hat = f_hat - Hhat u_hat on `level` as the V-cycle of a mixed-precision
 * context forms it: FP32 vectors (f_hat, u_hat, r_hat: condensed size of the
 * level), the arithmetic of the context's precision (FP64 for SEMMG_MIXED,
 * _TC and _BF16; float-float on the levels with p >= 12 for SEMMG_MIXED_FF and
 * _FF_TC, FP64 below; FP32 for SEMMG_MIXED_FP32 and _FP32_TC), the result
 * rounded once to FP32.  r_hat may alias f_hat, not u_hat.
 * SEMMG_ERR_UNSUPPORTED for an FP64 context. */
int semmg_residual_cycle(semmg_ctx* ctx, int level, const float* f_hat, const float* u_hat, float* r_hat,
                         void* stream);

/* du_hat = Smoother(r_hat): Algorithm 2 around Algorithm 1 on the stars of all
 * (n1+1)(n2+1)(n3+1) vertices of the level (Sec. 3.2), level >= 1; with
 * opts.smoother = SEMMG_SMOOTHER_ELEMENT(_MULT) the element-centred blocks of
 * Sec. 3.4 instead: per element the 3x3x3-element block, condensed to the six
 * planes through the element's faces (n_E = 3p - 1 points a side) and inverted
 * by the block's fast diagonalisation restricted to those planes (73 n_E^3
 * operations), outputs weighted as the option says.  dtype SEMMG_F64 or SEMMG_F32
 * gives the element type of both vectors and the arithmetic.  Overwrites du_hat
 * (zero on the Dirichlet boundary). */
int semmg_smooth(semmg_ctx* ctx, int level, int dtype, const void* r_hat, void* du_hat, void* stream);

/* coarse = J^T fine: restriction from level `level` (>= 1) to level-1, the exact
 * transpose of the embedded interpolation (Sec. 4.1).  Overwrites coarse. */
int semmg_restrict(semmg_ctx* ctx, int level, int dtype, const void* fine, void* coarse, void* stream);

/* fine += J coarse: prolongation from level-1 to level `level` (>= 1), the
 * embedded 1D interpolation tensor product restricted to the skeleton. */
int semmg_prolong_add(semmg_ctx* ctx, int level, int dtype, const void* coarse, void* fine, void* stream);

/* u_hat0 = Hhat_0^{-1} f_hat0 on level 0, exact, FP64: the full degree-p0
 * system with right-hand side (f_hat0 on the skeleton, 0 in the element
 * interiors) solved by global fast diagonalisation; its skeleton part is the
 * condensed solution (Sec. 3.1 embedding argument). */
int semmg_coarse_solve(semmg_ctx* ctx, const double* f_hat0, double* u_hat0, void* stream);

/* One V-cycle of Algorithm 3 on the finest level: u_hat <- MultigridCycle(u_hat, f_hat),
 * computed as u_hat + MultigridCycle(0, f_hat - Hhat u_hat) (equal in exact
 * arithmetic); the inner cycle runs in the context's precision. */
int semmg_vcycle(semmg_ctx* ctx, double* u_hat, const double* f_hat, void* stream);

/* f_hat = F_B - H_BI H_II^{-1} F_I with F = M f, M the assembled GLL mass and
 * f_nodal the right-hand side at every GLL node (Algorithm 4, condensation). */
int semmg_condense_rhs(semmg_ctx* ctx, const double* f_nodal, double* f_hat, void* stream);

/* u_nodal = (u_hat, H_II^{-1}(F_I - H_IB u_hat)) (Algorithm 4, recovery); writes
 * every node of u_nodal (0 on the Dirichlet boundary). */
int semmg_recover(semmg_ctx* ctx, const double* f_nodal, const double* u_hat, double* u_nodal,
                  void* stream);

/* Algorithm 4 (opts.solver = SEMMG_SOLVER_MG): condense, V-cycles from
 * u_hat = 0 until ||r|| <= rtol ||r_0|| (Euclidean norm over the condensed
 * unknowns, checked on the host after each cycle: one 8-byte device-to-host
 * copy per cycle), recover.
 * Algorithm 5 (opts.solver = SEMMG_SOLVER_KMG): the same with the inexact
 * preconditioned CG iteration of Sec. 4.1 in place of the plain cycle loop:
 * z = MultigridCycle(0, r), gamma = z.r, gamma0 = z.s, beta = (gamma -
 * gamma0) / delta, p = beta p + z, q = Hhat p, alpha = gamma / q.p, s = r,
 * u += alpha p, r -= alpha q; the stopping test uses this updated residual.
 * All of it in FP64 except the V-cycle in the mixed form; one Hhat
 * application per iteration, as in Algorithm 4.
 * f_nodal and u_nodal are device nodal arrays of the finest level.  info may
 * be NULL; info->iters counts iterations (V-cycles).  Returns
 * SEMMG_ERR_NOT_CONVERGED after max_iter iterations (u_nodal still holds the
 * last iterate), SEMMG_ERR_NONFINITE on a NaN/Inf residual norm,
 * SEMMG_ERR_DIVERGED as soon as ||r|| > 1e3 ||r_0|| (the iteration is not
 * contracting: a wrong operator, data or option, not a slow start; the factor
 * is set by semmg_set_guards), SEMMG_ERR_TIMEOUT when a tensor-core wait of
 * the smoother ran out during the solve.
 * Each iteration runs as one CUDA graph launch on `stream`: the first call
 * captures it on a stream the context owns (re-captured after semmg_autotune,
 * semmg_set_launch or a change of semmg_set_timing); results are bitwise those
 * of launching the kernels one by one. */
int semmg_solve(semmg_ctx* ctx, const double* f_nodal, double* u_nodal, double rtol,
                semmg_info* info, void* stream);

/* semmg_solve with inhomogeneous Dirichlet data (Sec. 5.2: u = g on the
 * Dirichlet faces).  g_nodal is a device nodal array of the finest level read
 * at the nodes on Dirichlet faces only (its other entries are ignored; it may
 * alias u_nodal).  Lifting: the iteration starts from u_hat = E g (see
 * semmg_pack_dirichlet), so r_0 = f_hat - Hhat E g carries the boundary data;
 * the V-cycle corrections vanish on the boundary slots, and the recovery reads
 * them, so u_nodal = g on the Dirichlet faces.  Same options, info and return
 * codes as semmg_solve; with g = 0 the result equals semmg_solve's. */
int semmg_solve_dirichlet(semmg_ctx* ctx, const double* f_nodal, const double* g_nodal, double* u_nodal,
                          double rtol, semmg_info* info, void* stream);

/* semmg_solve with HOST nodal arrays: copies f to the device, solves, and
 * synchronises `stream` before returning.  u goes back by a copy, or, when
 * u_host is page-locked host memory (cudaHostAlloc / cudaHostRegister), is
 * written by the unpack and recovery kernels through its device mapping (no
 * copy after the solve). */
int semmg_solve_host(semmg_ctx* ctx, const double* f_host, double* u_host, double rtol,
                     semmg_info* info, void* stream);

/* ------------------------------------------------------------------ batched form
 * Many independent solves (each its own context: any mesh, p, lambda,
 * precision) captured once into one CUDA graph and launched with one call.
 * Each solve is a branch of the graph: condensation, then a device-side loop
 * (a conditional WHILE node) of V-cycle, FP64 residual and norm (or one
 * Algorithm 5 iteration, per the context's opts.solver), whose check kernel
 * ends the loop when ||r|| <= rtol ||r_0|| or after max_iter iterations,
 * then interior recovery.  Branches are independent, so solves run
 * concurrently; no host round trip happens between cycles (Algorithm 4 with
 * the stopping test of Sec. 5.2 evaluated on the device).
 *
 * semmg_batch_create captures the graph: f[i] and u[i] are device nodal
 * arrays of context i that the graph keeps using (refill f[i] in place to
 * solve again).  The contexts must stay alive and must not be used by other
 * calls while a batch launch runs.  Allocates a small control block.
 * semmg_batch_solve launches the graph on `stream`, waits for it, and fills
 * infos[0..nb-1] (NULL allowed); it returns SEMMG_OK when every solve
 * converged, else the first non-zero status.
 * semmg_batch_create_dirichlet is the same with Dirichlet data per solve:
 * g_nodal[i] (device nodal array of context i, or NULL for homogeneous data;
 * g_nodal itself may be NULL) is read as semmg_solve_dirichlet reads it.
 * semmg_batch_graph_nodes reports the node count of the captured top-level
 * graph (kernel and memset nodes plus one conditional node per solve). */
typedef struct semmg_batch semmg_batch;
int semmg_batch_create(semmg_ctx* const* ctxs, int nb, const double* const* f_nodal, double* const* u_nodal,
                       double rtol, void* stream, semmg_batch** out);
int semmg_batch_create_dirichlet(semmg_ctx* const* ctxs, int nb, const double* const* f_nodal,
                                 const double* const* g_nodal, double* const* u_nodal, double rtol, void* stream,
                                 semmg_batch** out);
int semmg_batch_solve(semmg_batch* batch, semmg_info* infos, void* stream);
int semmg_batch_graph_nodes(const semmg_batch* batch, int64_t* nodes);
void semmg_batch_destroy(semmg_batch* batch);

/* ------------------------------------------------------------------ launch autotuning
 * For every level of the context, times a few launch shapes of the star
 * smoother (vertex-star contexts only) and of the element Schur kernel -- the
 * shared-memory budget per block (which decides which work arrays stay on
 * chip and how many blocks share an SM), the threads per block and the
 * register budget per thread (64 or 128, two builds of each kernel); the
 * Schur kernel is timed within a whole operator application -- on the
 * context's own buffers, and keeps the fastest.  Every shape computes bitwise the same
 * result; only the time changes.  Choices are cached per process by (kernel, element size,
 * degree, number of elements) and reused by later contexts without timing.  Synchronises the
 * stream; call it before capturing a batch. */
int semmg_autotune(semmg_ctx* ctx, void* stream);
/* Launch shape in use for `kernel` (0 = star smoother, 1 = element Schur
 * kernel) at `level` in element type dtype (SEMMG_F64 / SEMMG_F32):
 * threads per block, dynamic shared memory, blocks, and the register budget
 * per thread of the kernel build that runs (64 or 128).  On the levels where
 * a tensor-core form runs the FP32 star smoother on the tensor cores, the
 * shape of that kernel (which autotuning leaves as it is). */
int semmg_get_launch(const semmg_ctx* ctx, int level, int kernel, int dtype, int* block, int* smem_bytes, int* grid,
                     int* max_regs);
/* Pin the launch shape of `kernel` at `level` in dtype: a shared-memory budget
 * per block (work arrays that do not fit go to the context's global work
 * memory), threads per block (256 or 512) and registers per thread (64 or
 * 128); the blocks per launch follow from those.  For reproducing a tuned
 * configuration without timing, and for tests.  SEMMG_ERR_INVALID_ARG on a
 * bad value, SEMMG_ERR_UNSUPPORTED when the shape does not fit the context's
 * work memory (the shape in use is then unchanged). */
int semmg_set_launch(semmg_ctx* ctx, int level, int kernel, int dtype, int smem_cap_bytes, int block, int max_regs);

/* ------------------------------------------------------------------ no-allocation smoothing
 * The paper has no counterpart to this entry point; it exists for callers of
 * this library that must not allocate device memory while they work -- for
 * example code running under a memory manager that has already claimed the
 * device for its own pool, or a host thread that cannot afford the
 * device-wide synchronisation cudaMalloc and cudaFree may cause.
 *
 * semmg_smooth_noalloc computes exactly what semmg_smooth computes (du_hat =
 * Smoother(r_hat) on `level`, bitwise the same result) with the same kernels:
 * the CUDA-core star kernel, or for dtype SEMMG_F32 on the levels where the
 * context's precision (SEMMG_MIXED_TC, SEMMG_MIXED_FP32_TC, SEMMG_MIXED_BF16, SEMMG_MIXED_FF_TC) puts the star
 * transforms on the tensor cores, the tensor-core star kernel.  It calls no
 * cudaMalloc, cudaFree or other allocating routine: the star output buffer and
 * the per-block work arrays come from one array of SEMMG_NOALLOC_SCRATCH_BYTES
 * compiled into the library, which every GPU that loads the library holds
 * until the process exits.  The context (its read-only tables) must have been
 * set up beforehand by code that was allowed to allocate; the caller passes
 * r_hat and du_hat as for semmg_smooth.
 *   - Every call looks the array's device address up for the current device
 *     (cudaGetSymbolAddress, no allocation).  The first lookup on a device may
 *     load the library's device code there: make the first call on each device
 *     before any stream capture.
 *   - Vertex-star smoother only: a context set up with an element-centred
 *     smoother returns SEMMG_ERR_UNSUPPORTED.
 *   - A level whose star output buffer (nstar * 3 * n_S^2 elements) plus one
 *     block's work arrays exceeds the array returns SEMMG_ERR_UNSUPPORTED,
 *     with the sizes in semmg_last_error(ctx); larger work arrays only lower
 *     the number of blocks that run at once.  So does a level without a
 *     usable star launch plan.
 *   - A tensor-core completion wait that runs out sets the context's device
 *     error flag, as in semmg_smooth; the next semmg_solve clears it.
 *   - Every call, on every context, shares the one array and it keeps the
 *     last call's contents; each call writes every scratch entry it later
 *     reads, so nothing has to start at zero.  Calls whose executions overlap
 *     on the GPU (different streams, or different host threads) race on the
 *     array and give wrong results: order them on one stream. */
#define SEMMG_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
int semmg_smooth_noalloc(semmg_ctx* ctx, int level, int dtype, const void* r_hat, void* du_hat, void* stream);

/* ------------------------------------------------------------------ timing
 * Per-kernel-class timing with CUDA events recorded on the caller's stream
 * around every launch the context makes (off by default; a few microseconds
 * of host time per launch when on).  Each class also accumulates the
 * algorithmic work of its launches: SEMMG_K_STAR counts 37 n_S^3 flops per
 * star (Sec. 3.2 operation count of Algorithm 1); SEMMG_K_ELEM_SCHUR 73 m^3
 * per element, m = p-1 (six 2D transforms each way, expansion and
 * contraction); SEMMG_K_CONDENSE and SEMMG_K_RECOVER 12 p^4 + 25 p^3 per
 * element (Sec. 4.2); bytes are the compulsory reads and writes of each
 * launch's inputs and outputs. */
enum {
  SEMMG_K_STAR = 0,        /* Algorithm 1 on every star of a level */
  SEMMG_K_STAR_GATHER,     /* weighted star outputs summed per skeleton node */
  SEMMG_K_ELEM_SCHUR,      /* H_BI H_II^{-1} H_IB per element */
  SEMMG_K_ASSEMBLE,        /* H_BB line sums + element terms per skeleton node */
  SEMMG_K_TRANSFER,        /* restriction and prolongation */
  SEMMG_K_COARSE,          /* coarse fast diagonalisation */
  SEMMG_K_CONDENSE,        /* right-hand side condensation */
  SEMMG_K_RECOVER,         /* interior recovery */
  SEMMG_K_VECTOR,          /* copies, updates and norms */
  SEMMG_K_COUNT
};

typedef struct {
  double ms;         /* summed device time between the events around the launches */
  int64_t launches;  /* kernel launches of this class */
  double flops;      /* algorithmic flops of those launches */
  double bytes;      /* compulsory bytes of those launches */
  double xflops;     /* operations those launches execute, from the kernels' own loop trip counts (adds,
                        multiplies and divisions 1, fused multiply-adds 2); counted for the CUDA-core
                        star kernel (SEMMG_K_STAR), 0 for the other classes */
} semmg_kstat;

/* Switch timing on (1) or off (0); switching resets the statistics. */
int semmg_set_timing(semmg_ctx* ctx, int enable);
/* Statistics of one class since the last reset; synchronises the device
 * with the last recorded event. */
int semmg_get_kstat(semmg_ctx* ctx, int kind, semmg_kstat* out);
int semmg_reset_kstats(semmg_ctx* ctx);

/* ------------------------------------------------------------------ failure detection
 * Limits of the two failure checks of a context.
 *   divergence: semmg_solve (and the batched form) stops with
 *     SEMMG_ERR_DIVERGED as soon as ||r|| > divergence ||r_0|| after an
 *     iteration (default 1e3; > 0, +inf switches the check off).  A value below
 *     the first iteration's reduction makes the check trip on the first
 *     iteration, which is how the check itself is tested.
 *   tc_wait_cycles: budget, in SM clock cycles, of each completion wait of the
 *     tensor-core star smoother (default 4e9, about 2 s at 2 GHz; >= 0).  When
 *     a wait runs out the kernel sets the context's device error flag, waits
 *     (with the default budget) for the products it has in flight, frees its
 *     tensor memory and returns; semmg_solve then returns SEMMG_ERR_TIMEOUT.
 *     A budget of 0 makes every wait that is not already complete run out.
 * The device error flag is cleared at the start of every semmg_solve, so the
 * context stays usable.  Returns SEMMG_ERR_INVALID_ARG for a value out of range. */
int semmg_set_guards(semmg_ctx* ctx, double divergence, long long tc_wait_cycles);

/* Measured arithmetic peak of the current device in TFLOP/s: fused multiply-add
 * chains (eight independent chains per thread, four 256-thread blocks per SM),
 * dtype SEMMG_F64 or SEMMG_F32, one warm-up launch and one launch of about 10 ms
 * timed with CUDA events on `stream` (synchronises it).  The denominator of the
 * roofline fraction of ALU-bound kernels; no context needed. */
int semmg_peak_tflops(int dtype, double* tflops, void* stream);

/* Static message for an error code / last error message of a context. */
const char* semmg_strerror(int code);
const char* semmg_last_error(const semmg_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* SEMMG_H */
