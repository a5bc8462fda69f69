/*
 * aggmg.h - C ABI of libaggmg: agglomeration-based multigrid preconditioned
 * CG for the SIPG discontinuous-Galerkin monodomain model, on one NVIDIA
 * GB300 (sm_103a).
 *
 * The method (arXiv 2602.16312):
 *   - monodomain model and ionic models: Section 2 (Eq. monodomain, the
 *     FitzHugh-Nagumo model of Section 2.3.1, the Bueno-Orovio model of
 *     Section 2.3.2, Eq. BuenoOrovio);
 *   - SIPG forms a_h, m_h and penalty: Section 3; linear system
 *     A0 u^{n+1} = b with A0 = c M + A: Eq. fully_discrete;
 *   - nested agglomerated levels, inherited operators
 *     A_{l+1} = P^T A_l P: Section 5.1, Eq. inherited_matrices, Algorithm 3;
 *   - Chebyshev-accelerated Jacobi smoother, one V-cycle per PCG iteration,
 *     PCG warm-started from u^n: Section 6 (first paragraph), Section 3.1.
 *
 * Conventions for every call:
 *   - Handles are opaque and owned by the library (free with *_destroy).
 *   - `*_dev` arguments are device pointers owned by the caller (e.g. torch
 *     tensors); the library never frees or reallocates them. Vectors are
 *     float64, element-major: entry e*B + i is DoF i of element e, where
 *     B = (p+1)^d and i = i0 + (p+1) i1 [+ (p+1)^2 i2] indexes the tensor GLL
 *     nodes (x fastest). Coarse-level vectors use the caller's agglomerate
 *     ids in the same unit-major layout.
 *   - Host arrays passed to *_create / *_setup are copied; the caller may
 *     free them afterwards.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream). Device work
 *     is ordered on that stream; calls that return results to the host
 *     (agg_pcg_solve, agg_monodomain_step) synchronise it.
 *   - Every call returns an agg_status; nothing calls exit() or abort().
 *     agg_last_error() returns a message for the calling thread's last error.
 *   - A handle must not be used from two threads at once.
 */
#ifndef AGGMG_H
#define AGGMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  AGG_OK = 0,
  AGG_EINVAL = -1,        /* invalid argument (sizes, pointers, maps)          */
  AGG_ENOMEM = -2,        /* host or device allocation failed                  */
  AGG_ECUDA = -3,         /* a CUDA runtime call failed                        */
  AGG_ENOTSPD = -4,       /* a block or the coarsest matrix is not SPD         */
  AGG_ENOTCONV = -5,      /* PCG reached max_it before the tolerance           */
  AGG_ENAN = -6,          /* NaN or Inf in a residual norm                     */
  AGG_EUNSUPPORTED = -7   /* a combination the library does not provide        */
} agg_status;

typedef struct agg_mesh* agg_mesh_t;
typedef struct agg_hier* agg_hier_t;
typedef struct agg_sim* agg_sim_t;

/* ------------------------------------------------------------------ mesh
 * Conforming quadrilateral (dim 2) or hexahedral (dim 3) mesh with
 * multilinear element maps; corner c of an element sits at reference
 * coordinates ((c>>0)&1, (c>>1)&1, (c>>2)&1). Neighbouring elements share
 * vertex ids; a face of one element only is a boundary face (homogeneous
 * Neumann, Section 2.2). Element matrices use Gauss-Legendre quadrature with
 * p + 1 + quad_extra points per direction.
 *
 * SIPG penalty on an interior face F between K+ and K- (Section 3):
 *   sigma = C_pen * max(|F|/|K+|, |F|/|K-|) * n^T ((D+ + D-)/2) n,
 *   C_pen = p(p+1)                  if penalty_mode == 0 (the paper's alpha),
 *   C_pen = penalty_coeff * p^2     if penalty_mode == 1.
 */
typedef struct {
  int dim;                      /* 2 or 3                                        */
  int degree;                   /* p in 1..4                                     */
  int64_t n_vertices;
  int64_t n_elements;
  const double* vertices;       /* host [n_vertices][dim]                        */
  const int64_t* elements;      /* host [n_elements][2^dim] vertex ids           */
  const double* conductivity;   /* host [n_elements][dim][dim], symmetric SPD D  */
  int penalty_mode;             /* 0 or 1, see above                             */
  double penalty_coeff;
  int quad_extra;               /* >= 0; 1 gives p+2 points per direction        */
  int adjoint_data;             /* 1: also keep the per-element parts of A that
                                   the adjoint's conductivity gradient needs
                                   (volume form + 4 face blocks per neighbour;
                                   about 5x the stiffness memory)              */
  /* Optional conductivity parameters (not in the paper; for gradients with
   * respect to a coarse parameterisation): the assembly uses
   * theta[theta_map[e]] * D_e in place of D_e. theta: host [n_theta], each
   * finite and > 0; theta_map: host [n_elements] in [0, n_theta). NULL /
   * 0 = none. Both are copied. agg_theta_gradient reduces per-element
   * gradients to these parameters. */
  const double* theta;
  const int32_t* theta_map;
  int64_t n_theta;
} agg_mesh_desc;

/* Assembles, on the host in float64, the SIPG stiffness A and the element
 * mass blocks M_e (Section 3, Eq. matrices). Errors: AGG_EINVAL for bad sizes
 * or ids, a non-positive Jacobian or a non-conforming face. */
agg_status agg_dg_mesh_create(const agg_mesh_desc* desc, agg_mesh_t* out);
agg_status agg_dg_mesh_destroy(agg_mesh_t mesh);
/* n_dofs = n_elements * (p+1)^dim; n_faces = number of interior faces. */
agg_status agg_dg_mesh_info(agg_mesh_t mesh, int64_t* n_dofs, int64_t* n_faces);
/* Point evaluation of DG functions (sensors): for each of n host points
 * [n][dim], the containing element (Newton inversion of the element map) and
 * the B basis values there, so u_h(x_s) = sum_i weights[s][i] u[elem[s]*B+i].
 * Host arrays. AGG_EINVAL if a point lies outside the mesh. */
agg_status agg_dg_mesh_locate(agg_mesh_t mesh, int64_t n, const double* points, int64_t* elem,
                              double* weights);

/* ------------------------------------------------------------------ hierarchy */
enum { AGG_F64 = 0, AGG_F32 = 1, AGG_F32_BF16SMOOTH = 2 };

typedef struct {
  int n_levels;                  /* L >= 1 (1 = direct solve on level 0)        */
  const int32_t* const* agg_maps;/* L-1 host maps; map l sends every level-l unit
                                    to its level-(l+1) agglomerate in
                                    [0, N_{l+1}); every id must be used         */
  int smoother_degree;           /* Chebyshev degree (default 3)                 */
  int block_jacobi;              /* 1: (p+1)^d blocks (default); 0: point Jacobi */
  int lanczos_steps;             /* default 12                                   */
  double cheb_upper_safety;      /* lambda_max = safety * Ritz max (default 1.2) */
  double cheb_range;             /* lambda_min = lambda_max / range (default 20) */
  int vcycle_precision;          /* AGG_F64, AGG_F32 or AGG_F32_BF16SMOOTH       */
  int fine_operator;             /* V-cycle's level-0 operator: 0 assembled
                                    blocks; 1 matrix-free (the SIPG form and
                                    mass term evaluated from quadrature data
                                    with sum factorisation, Section 5.2); 1
                                    needs quadrilaterals with p <= 3 or
                                    hexahedra with p <= 3 whose neighbours
                                    list each shared face's corners in the
                                    same order, quad_extra 1 and a float32
                                    V-cycle, else AGG_EUNSUPPORTED. The outer
                                    CG always uses the assembled float64
                                    operator.                                */
  int coarse_persistent;         /* 1: run levels >= 1 and the coarsest solve
                                    of each V-cycle as one cooperative kernel
                                    with grid-wide barriers (hierarchies of 3
                                    or more levels, blocks of at most 32 DoFs;
                                    otherwise ignored); 0 (default): one kernel
                                    per level step. Same results bit for bit.
                                    On GB300 a grid barrier costs ~3 us against
                                    ~0.7 us between kernels of a CUDA graph,
                                    so 0 is faster.                           */
  int coarse_cluster;            /* 1: the smallest levels (from the first
                                    level of at most 16 x 1024 rows on, blocks
                                    of at most 32 DoFs) and the coarsest solve
                                    run as one kernel on a thread-block
                                    cluster of 16 (else 8) CTAs whose steps
                                    are separated by the cluster's hardware
                                    barrier; 0 (default): one kernel per level
                                    step. Same results bit for bit. Ignored
                                    with coarse_persistent = 1. Measured on
                                    GB300: within 0.3% of 0 in 2D, 1-2% slower
                                    in 3D.                                   */
  int coarse_operator;           /* 0 (default): inherited operators
                                    A_{l+1} = P^T A_l P (Eq. inherited_matrices,
                                    the paper's choice); 1: non-inherited ones
                                    (Section 5.1): c M_l + A_l assembled on the
                                    agglomerates by quadrature over the fine
                                    elements and the fine faces between
                                    agglomerates, with the level's box basis
                                    and the penalty C_pen max(|F|/|K+|,
                                    |F|/|K-|) n^T D n of the polytopic face F.
                                    Measured on the jittered square: more PCG
                                    iterations than 0 (19-21 against 14 at
                                    128^2).                                  */
} agg_mg_opts;

void agg_mg_opts_default(agg_mg_opts* opts);

/* Algorithm 3 on the host in float64 with A0 = mass_coeff * M + A: bounding
 * boxes of the agglomerates, prolongation blocks (nodal interpolation of the
 * Q_p bounding-box basis, Section 5.1), Galerkin operators
 * A_{l+1} = P^T A_l P (Eq. inherited_matrices), smoother blocks and their
 * inverses, Lanczos bounds, Cholesky factor of the coarsest operator; then
 * uploads everything to the current device in the requested precision and
 * captures the solver's CUDA graphs. The device must stay the same for the
 * handle's lifetime. Errors: AGG_EINVAL (maps), AGG_ENOTSPD, AGG_ENOMEM,
 * AGG_ECUDA. */
agg_status agg_mg_hierarchy_setup(agg_mesh_t mesh, double mass_coeff, const agg_mg_opts* opts,
                                  void* stream, agg_hier_t* out);
agg_status agg_mg_hierarchy_destroy(agg_hier_t hier);
/* Per level l: units[l], block nonzeros nnzb[l] (pass arrays of n_levels
 * entries or NULL), Chebyshev lambda_max[l] for l < L-1 (NULL allowed) and the
 * operator complexity sum_l nnz(A_l) / nnz(A_0). */
agg_status agg_hier_stats(agg_hier_t hier, int* n_levels, int64_t* units, int64_t* nnzb,
                          double* lambda_max, double* op_complexity);

/* ------------------------------------------------------------------ solve */
typedef struct {
  double rtol;     /* stop when ||r||_2 <= rtol ||r0||_2 ...                     */
  double atol;     /* ... or ||r||_2 <= atol                                     */
  int max_it;      /* limit on products A0 p; reaching it gives AGG_ENOTCONV     */
  int flexible;    /* 1: Polak-Ribiere beta (safe with the float32 V-cycle)      */
} agg_pcg_opts;

typedef struct {
  int iterations;  /* number of products A0 p                                     */
  double r0_norm;
  double r_norm;
  int status;      /* agg_status of the solve                                     */
} agg_pcg_result;

/* PCG on A0 x = b preconditioned by one V-cycle per iteration (Section 6),
 * x_dev holds the initial guess on entry and the solution on return. The
 * outer recurrence, dot products and x are float64 in every precision form.
 * Synchronises `stream`. Returns AGG_ENOTCONV / AGG_ENAN as the result's
 * status too. */
agg_status agg_pcg_solve(agg_hier_t hier, const double* b_dev, double* x_dev,
                         const agg_pcg_opts* opts, agg_pcg_result* res, void* stream);
/* y = A_l x with the level's stored operator (float64 on level 0 always;
 * levels >= 1 in the V-cycle precision, converted from/to float64).
 * level = -1: the V-cycle's level-0 operator in the V-cycle precision (the
 * matrix-free one when fine_operator = 1).
 * level = -2: the level-0 operator evaluated matrix-free in float64 (the
 * quadrature data of fine_operator = 1 kept in float64; built on the first
 * such call; the mesh kinds of fine_operator = 1, in any V-cycle precision).
 * It is a measured alternative to the assembled float64 operator of the
 * outer CG, which keeps the assembled one (see agg_profile_kernel id 5).
 * The mesh must stay alive while hierarchies built from it exist. */
agg_status agg_operator_apply(agg_hier_t hier, int level, const double* x_dev, double* y_dev,
                              void* stream);
/* z = B r: one V-cycle of the preconditioner (Section 6). */
agg_status agg_vcycle_apply(agg_hier_t hier, const double* r_dev, double* z_dev, void* stream);

/* ------------------------------------------------------------------ allocation-free product
 * agg_operator_apply_static: the same product y = A_l x as agg_operator_apply
 * (same operator, same kernels, same results), for callers that must not
 * allocate device memory at the time of the call, such as an embedding that
 * fixes its device-memory budget at start-up.
 * It has no counterpart in the paper: it only changes where the two
 * temporary, unit-permuted copies of x and y live.
 *
 * Scratch: one file-scope device array of 2 x AGG_STATIC_APPLY_MAX_ENTRIES
 * doubles (16 MiB), which every GPU that loads the library holds until the
 * process exits. The call calls no cudaMalloc, cudaFree or other allocating
 * routine. Levels 0 .. n_levels-2 only; a level whose padded vector length
 * ((units rounded up to 32) * (p+1)^d) exceeds AGG_STATIC_APPLY_MAX_ENTRIES
 * returns AGG_EINVAL. The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress, once per device, with that device current).
 * The address is kept for
 * the life of the process, so resetting the device (cudaDeviceReset) or
 * destroying its primary context after the first call is not supported
 * while the library stays loaded. The array is shared by all calls and keeps
 * the last call's contents; nothing in it has to start at zero: every entry
 * that contributes to y is written earlier in the same call, and the padded
 * lanes of the last 32-unit slice, which may read stale entries, only feed
 * padded outputs that are never copied to y. Calls that overlap on the GPU
 * (two streams, or two threads) race on the array: order them on one
 * stream. */
#define AGG_STATIC_APPLY_MAX_ENTRIES (1LL << 20)
agg_status agg_operator_apply_static(agg_hier_t hier, int level, const double* x_dev, double* y_dev,
                                     void* stream);

/* ------------------------------------------------------------------ agglomeration
 * R*-tree agglomeration (Section 4.1, Algorithms 1 and 2), on the host. The
 * elements' axis-aligned bounding boxes (of their corner vertices) are
 * inserted in element order into an R*-tree holding at most max_entries
 * (>= 4) entries per node, with the insertion algorithm of Beckmann et al.
 * (choose-subtree by least overlap enlargement just above the leaves and
 * least area enlargement higher up; one forced reinsert of the 30% farthest
 * entries per tree level and inserted element; split on the axis of least
 * margin sum at the distribution of least overlap; minimum fill 40%). The
 * nodes of height h agglomerate the elements below them; heights 0, 1, ...
 * give nested levels: maps[0][e] = leaf node of element e, and for k >= 1
 * maps[k][i] = parent of node i of height k-1, nodes numbered depth-first
 * from the root. maps: n_maps caller-owned host arrays of at least
 * n_elements int32 each (maps[k] is filled up to n_units[k-1] entries,
 * maps[0] up to n_elements); n_units[k] receives the units of level k+1;
 * tree_levels (may be NULL) the number of node levels. The result can be
 * passed as agg_mg_opts.agg_maps with n_levels = n_maps + 1. Errors:
 * AGG_EINVAL for max_entries < 4, n_maps above the tree's levels or NULL
 * arrays (with n_maps = 0 the call only reports tree_levels). */
agg_status agg_rtree_agglomerate(agg_mesh_t mesh, int max_entries, int n_maps, int32_t* const* maps,
                                 int64_t* n_units, int* tree_levels);

/* ------------------------------------------------------------------ ionic models */
typedef enum { AGG_FHN = 0, AGG_ALIEV_PANFILOV = 1, AGG_BUENO_OROVIO = 2 } agg_ionic_model;

/* Bueno-Orovio (Section 2.3.2, Eq. BuenoOrovio; values in the paper's
 * appendix table). Names follow the paper: tau1p = tau_1', tau1pp = tau_1'',
 * tau1plus = tau_1^+, tau2inf = tau_2^inf, tauo_p = tau_o', tauso_pp =
 * tau_so'', winf_star = w_inf^*, V1m = V_1^-, Vhat = V^, and so on; uo is the
 * reference potential of the I_so drift term (u - uo). With H_z0 the unit
 * step at z0 (1 for u >= z0) and H^k_z0 = (1 + tanh(k (u - z0)))/2, three
 * gates evolve as dw_i/dt = (b_i - a_i) w_i + a_i w_i^inf:
 *   a0 = (1 - H_V1)/(H_V1m (tau1pp - tau1p) + tau1p), b0 = -H_V1/tau1plus,
 *   w0^inf = 1 - H_V1m;
 *   a1 = (1 - H_V2)/(H^k2_V2m (tau2pp - tau2p) + tau2p), b1 = -H_V2/tau2plus,
 *   w1^inf = H_Vo (winf_star - 1 + u/tau2inf) + 1 - u/tau2inf;
 *   a2 = 1/(H_V2 (tau3pp - tau3p) + tau3p), b2 = 0, w2^inf = H^k3_V3;
 * and I_ion = -H_V1 (u - V1)(Vhat - u) w0/taufi
 *           + (1 - H_V2)(u - uo)/(H_Vo (tauo_pp - tauo_p) + tauo_p)
 *           + H_V2/(H^kso_Vso (tauso_pp - tauso_p) + tauso_p) - H_V2 w1 w2/tausi. */
typedef struct {
  double tau1p, tau1pp, tau1plus, tau2p, tau2pp, tau2plus, tau2inf, tau3p, tau3pp;
  double taufi, tauo_p, tauo_pp, tauso_p, tauso_pp, tausi;
  double k2, k3, kso, winf_star;
  double V1, V1m, V2, V2m, V3, Vhat, Vo, Vso, uo;
} agg_bueno_orovio_params;

/* FitzHugh-Nagumo (Section 2.3.1): I = k u (u-a)(u-1) + w, H = eps (u - gamma w).
 * Aliev-Panfilov (not in the paper; published 1996 form):
 *   I = k u (u-a)(u-1) + u w, H = (eps + mu1 w/(u+mu2)) (-w - k u (u-a-1)).
 * Bueno-Orovio: the fields of `bo` (k ... mu2 unused).
 * Gating state: FitzHugh-Nagumo and Aliev-Panfilov have one gate per DoF,
 * Bueno-Orovio three; an array w of n DoFs holds the gates one after the
 * other, w[g * n + i] (gate g of DoF i). */
typedef struct {
  int model;
  double k, a, eps, gamma, mu1, mu2;
  agg_bueno_orovio_params bo;
} agg_ionic_params;

/* w <- w + dt H(u, w) at n DoFs (forward Euler; Section 3.1, first bullet).
 * w_dev holds n_gates * n values (gate-major, see above). */
agg_status agg_ionic_update(const agg_ionic_params* prm, double dt, int64_t n, const double* u_dev,
                            double* w_dev, void* stream);

/* ------------------------------------------------------------------ time stepping */
typedef struct {
  double dt, chi_m, c_m;          /* mass coefficient: chi_m c_m / dt (scheme 0),
                                     3 chi_m c_m / (2 dt) (scheme 1)             */
  agg_ionic_params ionic;
  const double* iapp_mask_dev;    /* [n_dofs] nodal stimulus mask (copied)        */
  double iapp_value;              /* I_app = iapp_value * mask for the first      */
  int iapp_steps;                 /* iapp_steps steps, zero afterwards            */
  agg_pcg_opts pcg;
  int scheme;                     /* 0 IMEX backward Euler, 1 BDF2 (see below)    */
} agg_sim_opts;

/* One step n -> n+1 (Section 3.1, ionic current interpolation).
 * scheme 0, backward-Euler form of Eq. fully_discrete:
 *   w^{n+1} = w^n + dt H(u^n, w^n)
 *   b = M (c u^n + I_app(t_{n+1}) - chi_m I_ion(u^n, w^{n+1})),  c = chi_m c_m/dt
 * scheme 1, BDF2 with the extrapolation U* = 2u^n - u^{n-1} (Eq. fully_discrete):
 *   W* = 2w^n - w^{n-1}, w^{n+1} = (4w^n - w^{n-1})/3 + (2dt/3) H(U*, W*)
 *   b = M (chi_m c_m (4u^n - u^{n-1})/(2dt) + I_app(t_{n+1}) - chi_m I_ion(U*, w^{n+1}))
 *   the history (u^{n-1}, w^{n-1}) is kept by the handle; at the first step
 *   (and after agg_monodomain_set_clock) it is started at second order:
 *   u^{-1} = u - dt u', chi_m c_m u' = I_app - chi_m I_ion(u, w) - M^{-1} A u,
 *   w^{-1} = w - dt H(u, w).
 * Both: A0 u^{n+1} = b by PCG warm-started from u^n. */
agg_status agg_monodomain_create(agg_hier_t hier, const agg_sim_opts* opts, agg_sim_t* out);
/* Advances n_steps steps in place on u_dev ([n_dofs]) and w_dev
 * ([n_gates][n_dofs], gate-major as for agg_ionic_update); the
 * stimulus clock is the handle's step counter (starts at 0). iters_out: host
 * array of n_steps PCG iteration counts, or NULL. Synchronises `stream`. */
agg_status agg_monodomain_step(agg_sim_t sim, int n_steps, double* u_dev, double* w_dev,
                               int* iters_out, void* stream);
agg_status agg_monodomain_set_clock(agg_sim_t sim, int64_t step);
/* Discrete adjoint of one step n -> n+1 (not in the paper; the reverse of
 * agg_monodomain_step for gradients of a loss of the states). Inputs: the
 * states u_n, w_n at the start of the step and u_np1 after it; ubar, wbar =
 * dL/du^{n+1}, dL/dw^{n+1} on entry, overwritten with dL/du^n, dL/dw^n:
 *   lambda = K^{-1} ubar (same MG-PCG and options as the forward solve,
 *   zero initial guess, K = c M + A symmetric), q = M lambda,
 *   w~ = wbar - chi I_w(u^n, w^{n+1}) q,
 *   ubar <- q (c - chi I_u(u^n, w^{n+1})) + dt H_u(u^n, w^n) w~,
 *   wbar <- w~ (1 + dt H_w(u^n, w^n)).
 * grad_logD_dev [n_elements] accumulates, per element e, the derivative of L
 * with respect to log s_e for D_e -> s_e D_e: -lambda^T A_e u^{n+1}, A_e the
 * part of A built with D_e (element-local volume form and e's share of its
 * face forms). Needs a mesh created with adjoint_data = 1 and a one-gate
 * ionic model (AGG_EUNSUPPORTED for Bueno-Orovio). Synchronises `stream`;
 * returns the adjoint solve's status. */
agg_status agg_monodomain_adjoint_step(agg_sim_t sim, const double* u_n_dev, const double* w_n_dev,
                                       const double* u_np1_dev, double* ubar_dev, double* wbar_dev,
                                       double* grad_logD_dev, void* stream);
agg_status agg_monodomain_destroy(agg_sim_t sim);
/* Chain rule from per-element log-conductivity gradients (the grad_logD_dev
 * of agg_monodomain_adjoint_step, caller's element order) to the mesh's
 * conductivity parameters: theta_grad_dev[k] += sum_{e: theta_map[e] = k}
 * grad_logD_dev[e] / theta[k], since D_e = theta_k D0_e gives d log s_e =
 * d theta_k / theta_k. On the device, one warp per parameter summing its
 * elements in increasing element order (deterministic). Device arrays of
 * n_elements and n_theta doubles, on the hierarchy's device. AGG_EINVAL if the
 * hierarchy's mesh has no theta. Ordered on `stream`; does not synchronise. */
agg_status agg_theta_gradient(agg_hier_t hier, const double* grad_logD_dev, double* theta_grad_dev,
                              void* stream);

/* ------------------------------------------------------------------ instrumentation
 * Kernel ids: 0 fine float64 SpMV y = A0 x (the outer CG's operator),
 * 1 fine Chebyshev step in the V-cycle precision (SpMV + residual + block
 * inverse + two axpys), 2 fine residual + restriction, 3 fine prolongation.
 * agg_profile_kernel launches the kernel `reps` times on the hierarchy's own
 * work buffers (valid after any solve or V-cycle) on `stream`, so a caller
 * can time it with events; agg_kernel_cost gives its algorithmic HBM bytes
 * (every matrix, block and vector entry read or written once) and flops per
 * launch. Kernels 1-3 need n_levels >= 2 (else AGG_EUNSUPPORTED).
 * Id 5 is the level-0 operator evaluated matrix-free in float64 (the
 * operator of agg_operator_apply level -2, built by the first call), the
 * same product as id 0 from quadrature data instead of stored blocks; its
 * flops are counted as id 0's (two per stored entry of the assembled
 * operator), so the two ids compare as the same work.
 * agg_kernel_cost also takes id 4: one iteration of the solve body (float64
 * SpMV, CG update, one V-cycle over every level, z and p updates), the sum
 * of its launches' algorithmic bytes and flops, counting the float32 copy of
 * r and the flexible (r, z_old) read in the reduced-precision forms;
 * agg_profile_kernel rejects it (AGG_EINVAL). */
agg_status agg_profile_kernel(agg_hier_t hier, int kernel, int reps, void* stream);
/* Kernel launches of the solver's work, for launch accounting: per V-cycle,
 * per PCG iteration (float64 SpMV, CG update, V-cycle, dot product, p update,
 * loop control) and per solve set-up (the initial residual, its norm, the
 * first V-cycle and p). *persistent is 1 when levels >= 1 and the coarsest
 * solve run as one persistent kernel (hierarchies of 3 or more levels with
 * blocks of at most 32 DoFs), 0 when they run as separate kernels per level
 * and step. *cluster_level (may be NULL) is the first level run by the
 * cluster kernel of agg_mg_opts.coarse_cluster, or -1 when none runs;
 * *cluster_ctas (may be NULL) its CTAs. Host only; no device work. */
agg_status agg_hier_launches(agg_hier_t hier, int* per_vcycle, int* per_iteration, int* per_setup,
                             int* persistent, int* cluster_level, int* cluster_ctas);
agg_status agg_kernel_cost(agg_hier_t hier, int kernel, double* bytes, double* flops);

/* ------------------------------------------------------------------ host inspection
 * Host-only access to the float64 set-up (no device needed), for checking
 * the assembly and Algorithm 3 against an independent implementation.
 * agg_dg_mesh_copy `what`: 0 stiffness row pointers (int64, n_elements+1),
 * 1 block columns (int32, nnzb), 2 blocks (float64, nnzb*B*B, row-major
 * blocks), 3 element mass blocks (float64, n_elements*B*B), 4 element
 * volumes (float64, n_elements), 5 element volume forms (float64,
 * n_elements*B*B) and 6 per-block face parts (float64, nnzb*4*B*B: for block
 * k of row e with column n, the (ee, en, ne, nn) blocks of the face terms
 * built with D_e), both only with adjoint_data. The stiffness excludes the
 * mass term. */
agg_status agg_dg_mesh_copy(agg_mesh_t mesh, int what, void* dst);
agg_status agg_dg_mesh_nnzb(agg_mesh_t mesh, int64_t* nnzb);

typedef struct agg_host_hier* agg_host_hier_t;
/* Runs the host part of agg_mg_hierarchy_setup (same arguments, no upload). */
agg_status agg_host_hierarchy_build(agg_mesh_t mesh, double mass_coeff, const agg_mg_opts* opts,
                                    agg_host_hier_t* out);
agg_status agg_host_hierarchy_destroy(agg_host_hier_t hh);
/* Level l: units, block nonzeros, lambda_max (0 on the coarsest). */
agg_status agg_host_hierarchy_level(agg_host_hier_t hh, int level, int64_t* n_units, int64_t* nnzb,
                                    double* lambda_max);
/* Copies level data in the library's internal unit order. `what`:
 * 0 perm (int64, n: internal index -> caller's id), 1 row pointers (int64,
 * n+1), 2 block columns (int32, nnzb, internal indices), 3 blocks (float64,
 * nnzb*B*B row-major), 4 smoother block inverses (float64, n*B*B),
 * 5 prolongation blocks to level l+1 (float64, n*B*B, P[u][i][j] =
 * coarse basis j at node i), 6 parent (int32, n, internal index on l+1). */
agg_status agg_host_hierarchy_copy(agg_host_hier_t hh, int level, int what, void* dst);

const char* agg_status_string(int status);
const char* agg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* AGGMG_H */
