/*
 * romb.h -- C ABI of the GB300 library for the ROM-accelerated BDDC solver of
 * unfitted p-FEM level-set lattices (Bonilla Moreno, Guarino, Antolin,
 * arXiv 2604.09113).
 *
 * The library owns every device buffer it needs; the caller passes plain host
 * (or, where stated, device) pointers and sizes.  All calls enqueue work on the
 * context's CUDA stream.  Calls that return data to host memory synchronise that
 * stream before returning.  Every call returns a romb_status; a failed call
 * leaves the context usable (unless the status is ROMB_E_CUDA after a sticky
 * device error).
 *
 * Call order (anything else returns ROMB_E_STATE):
 *   romb_create -> romb_train_load (one per level-set family)
 *     -> romb_assemble | romb_assemble_host_K -> romb_factor
 *     -> romb_bddc_solve (any number of times) -> romb_destroy.
 *
 * Conventions shared by every call
 *  - Lattice of nx*ny cells, cell c = cx + nx*cy, each cell the parametric unit
 *    square (Sec. 2.1.1) mapped by a tensor-product Lagrange map of order m on
 *    equispaced nodes a/m, a = 0..m.  The map control points of all cells form
 *    one grid of (m*nx+1) x (m*ny+1) points g = gx + (m*nx+1)*gy, so shared
 *    edges have shared maps (Eq. GEO untrimmed compatibility).
 *  - Thresholds mu[c][0..3] at the bottom-left, bottom-right, top-left and
 *    top-right corners, interpolated bilinearly (Sec. 2.1.2).
 *  - Families: 0 circle hole (solid where |xi - (1/2,1/2)| > mu(xi)),
 *    1 solid cross (solid where min(|xi1 - 1/2|, |xi2 - 1/2|) < mu(xi)).
 *  - Cell basis: degree-p tensor polynomials on GLL nodes (Sec. 2.2.2) or
 *    Bernstein polynomials; local node k = a + (p+1) b, local DoF 2k + i.
 *  - Displacements are returned on the global node grid (p*nx+1) x (p*ny+1),
 *    node n = gx + (p*nx+1) gy, as u[n][2] (for the Bernstein basis these are
 *    the basis coefficients at the same grid positions).
 *  - Lattice edges 0 left, 1 right, 2 bottom, 3 top.
 */
#ifndef ROMB_H
#define ROMB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct romb_ctx romb_ctx;

typedef enum {
  ROMB_OK = 0,
  ROMB_E_ARG = -1,            /* invalid argument or unsupported size          */
  ROMB_E_CUDA = -2,           /* CUDA runtime error                            */
  ROMB_E_OOM = -3,            /* device allocation failed or budget exceeded   */
  ROMB_E_OUT_OF_BOX = -4,     /* a threshold lies outside its ROM's box        */
  ROMB_E_BAD_MAP = -5,        /* det J <= 0 at an interpolation node           */
  ROMB_E_NOT_SPD = -6,        /* non-positive pivot in a local or coarse factor */
  ROMB_E_NOT_CONVERGED = -7,  /* PCG reached maxit (u_out holds the last iterate) */
  ROMB_E_NAN = -8,            /* non-finite value detected                     */
  ROMB_E_FORMAT = -9,         /* malformed ROM file                            */
  ROMB_E_STATE = -10,         /* call out of order                             */
  ROMB_E_SCRATCH = -11        /* problem too large for the fixed scratch of    */
                              /* romb_compliance_grad_noalloc                  */
} romb_status;

typedef enum {
  ROMB_FP64 = 0,        /* assembly contraction in FP64 on the CUDA cores          */
  ROMB_FP32_SPLIT = 1,  /* tcgen05 kind::tf32, 3-term hi/lo split, FP32 accumulate */
  ROMB_BF16_SPLIT = 2   /* tcgen05 kind::f16 (bf16), 4-part split, 10 products     */
} romb_precision;

typedef enum { ROMB_MEM_HOST = 0, ROMB_MEM_DEVICE = 1 } romb_mem;

/* Problem statement of Sec. 2.2.1: geometry (maps + level sets + thresholds),
 * material, loads and Dirichlet constraints.  Pointers follow `mem`: host
 * memory (copied to the device during the call) or device memory on the
 * context's device (read in place, must stay valid until romb_factor returns). */
typedef struct {
  int nx, ny;              /* cells per direction, >= 1                          */
  int p;                   /* polynomial degree of the cell basis, 3..8          */
  int map_order;           /* m, 1..4                                            */
  int basis;               /* 0 GLL Lagrange, 1 Bernstein                        */
  int mem;                 /* romb_mem of every pointer below (and of u_out)     */
  const double* ctrl;      /* [(m*nx+1)*(m*ny+1)][2] map control points          */
  const double* mu;        /* [nx*ny][4] corner thresholds                       */
  const int32_t* family;   /* [nx*ny] family id of a loaded ROM                  */
  double E, nu;            /* Young modulus, Poisson ratio (plane stress)        */
  double rho;              /* alpha-stabilisation factor, Eq. (MOD stabilization) */
  unsigned dirichlet_mask; /* bit e: lattice edge e clamped (u = 0, strong)      */
  const double* traction;  /* [4][2] physical traction per unit length per edge, */
                           /* applied on the solid (conformal) part of the edge  */
  /* Layouts that are not a full rectangle of cells (the lattice wrench of
   * Sec. 5.2.2): the subdomains are the present cells of the nx x ny grid.
   * Edges that a present cell shares with an absent one are free boundary;
   * dirichlet_mask and traction act on the present cells' edges on the
   * grid's sides.  Per-cell results (romb_read, the per-cell flags) list the
   * present cells in increasing grid index c = cx + nx cy; mu and family
   * keep one entry per grid cell, absent ones unread; the nodal output keeps
   * the full grid, zero at nodes of no present cell.  The compliance
   * gradient needs the full rectangle (ROMB_E_STATE otherwise). */
  const uint8_t* cell_present;  /* [nx*ny] nonzero: cell present; NULL: all     */
  const uint8_t* edge_clamped;  /* [nx*ny][4] nonzero: edge e (0 left, 1 right, */
                                /* 2 bottom, 3 top) of that present cell clamped, */
                                /* end points included; NULL: none              */
} romb_lattice;

/* Create a context on `device`.  `cuda_stream` is a cudaStream_t owned by the
 * caller (NULL: the library creates its own).  mem_budget_bytes caps the
 * device memory the context may hold (0: no cap). */
romb_status romb_create(romb_ctx** ctx, int device, size_t mem_budget_bytes, void* cuda_stream);
void romb_destroy(romb_ctx* ctx);
const char* romb_strerror(romb_status s);

/* Load the trained reduced models of one family (Sec. 4.2, offline phase of
 * Sec. 4.4) and keep them resident in HBM.  File format: 128-byte header
 * "ROMBDDC1", int32 version (1 or 2), family, basis, p, q, r, n_r, n_k (1 or
 * 2), float64 lo, hi, int64 n_i; then float64 I_Pi[n_i]; then, for each of the
 * n_k^4 clusters of the box [lo,hi]^4 in cluster order (Sec. 4.2.1, see
 * romb_train_gpu_clustered): float64 U_r[n_r][n_i], A[n_r][(r+1)^4] (I_r at
 * the tensor GLL nodes of the cluster's box, node
 * g = g1 + (r+1)(g2 + (r+1)(g3 + (r+1) g4))), int64 magic[n_r]; version 2
 * adds to each cluster the reduced model of the force integrals J[e][s][k]
 * (edge e, edge node s, edge interpolation node k; see romb_set_load_form):
 * int64 n_f = 4 (p+1)(q+1) (tractions) or 4 (p+1)(q+1) + (p+1)^2 (q+1)^2
 * (tractions, then V[k][k3] for body forces), r_f <= 128, float64
 * U_f[r_f][n_f], A_f[r_f][(r+1)^4], int64 magic_f[r_f].  The trainers write
 * version 2.  At most 64 models are
 * resident (a family reloaded with another n_k takes new slots); a file that
 * fails to load leaves its family without models.  Assembly finds each
 * cell's cluster from its thresholds (FindCluster of Algorithm 5; an interior
 * subinterval boundary belongs to the upper cluster).
 * The fast-assembly vector is I[((k1*nB+k2)*nL+k3)*4 + 2*j1 + j2] (Eq. MDEIM I).
 * *family_out receives the file's family id.  Errors: ROMB_E_FORMAT. */
romb_status romb_train_load(romb_ctx* ctx, const char* rom_path, int* family_out);

/* Online assembly of every cell stiffness matrix (Algorithms 4 and 5):
 * theta = ((1-rho) I_r(mu), rho) from the MDEIM interpolation of the cell's
 * family, Chat at the (q+1)^2 interpolation nodes (Eq. FAST interpolation), and
 * the contraction K = sum_{j1 j2 k3} [U_r I_r (1-rho) + rho I_Pi] C.
 * prec = ROMB_FP64: everything in FP64.  The split forms interpolate theta in
 * double-float arithmetic (FP32 pairs, ~48-bit significands; within ~1e-13
 * of FP64) and run the contraction on the tensor cores with a compensated
 * double-float epilogue; K stays FP64 in memory in every form.
 * Errors: ROMB_E_OUT_OF_BOX, ROMB_E_BAD_MAP (per-cell flags via romb_stats). */
romb_status romb_assemble(romb_ctx* ctx, const romb_lattice* lat, romb_precision prec);

/* As romb_assemble, but with caller-supplied dense cell matrices
 * K[ncells][ndof][ndof] (ndof = 2 (p+1)^2, local DoF 2k+i; ncells = nx*ny,
 * or the present cells in increasing grid index), e.g. from full trimmed
 * quadrature (the unaccelerated baseline of Sec. 5.1). */
romb_status romb_assemble_host_K(romb_ctx* ctx, const romb_lattice* lat, const double* K);

/* BDDC set-up (Sec. 3): per cell the Cholesky factor of K_II and the Schur
 * complement S = K_UU - K_UI K_II^-1 K_IU, the constrained-Neumann factors of
 * Algorithm 2, the coarse basis Psi of Eq. (BDDC local basis), the stiffness
 * partition of unity D, the explicit fine operator D F D and the local coarse
 * matrix Psi^T S Psi; then the assembly of S_C and its sparse Cholesky factor
 * (nested dissection).  Errors: ROMB_E_NOT_SPD. */
romb_status romb_factor(romb_ctx* ctx);

/* PCG on the Schur system S u = f (Eq. BDDC system) preconditioned by
 * S_BDDC^-1 (Eq. BDDC preconditioner, Algorithm 1), x0 = 0, stopping when
 * ||r||_2 <= rtol ||f||_2; then interior recovery u_I = K_II^-1 (f_I - K_IU u).
 * traction_sets: [nrhs][4][2] (NULL: the lattice's traction, nrhs must be 1).
 * u_out: [nrhs][(p*nx+1)*(p*ny+1)][2] in the lattice's memory kind;
 * iters_out, relres_out: [nrhs] host arrays (may be NULL).
 * Errors: ROMB_E_NOT_CONVERGED (u_out holds the last iterate). */
romb_status romb_bddc_solve(romb_ctx* ctx, int nrhs, const double* traction_sets, double rtol,
                            int maxit, double* u_out, int* iters_out, double* relres_out);

/* Compliance c = f^T u of the last solve (first right-hand side) and its
 * gradient by the discrete adjoint (Sec. 6: the ROM makes the gradient
 * available): dc = 2 u^T df - sum_i u_i^T dK_i u_i, with dK_i through the
 * pulled-back tensor of Eq. (ELA constitutive) for the map control points and
 * through I_r(mu) of Algorithm 5 for the thresholds; cell matrices are
 * differentiated in their FP64 form.  The traction loads are differentiated
 * through the edge Jacobian only (their active interval is taken fixed in mu).
 * dc_dctrl: [(m*nx+1)*(m*ny+1)][2]; dc_dmu: [cells][4] (nullable);
 * dc_dR: [cells] = sum of the four dc/dmu_i (nullable; the derivative with
 * respect to a uniform per-cell threshold such as a hole radius).  Pointers
 * follow the lattice's memory kind.  Requires romb_assemble (not _host_K) and
 * a solve.  Errors: ROMB_E_STATE. */
romb_status romb_compliance_grad(romb_ctx* ctx, double* compliance, double* dc_dctrl, double* dc_dR,
                                 double* dc_dmu);

/* Size in bytes of the fixed device scratch of romb_compliance_grad_noalloc
 * (one array per device, 16 MiB). */
#define ROMB_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)

/* romb_compliance_grad for callers that cannot allocate device memory when
 * they need the gradient.  The paper has no counterpart of this call.
 *
 * Arguments, results, memory kinds and errors are those of
 * romb_compliance_grad, and the results are bitwise equal to its results.
 * romb_compliance_grad allocates its intermediate arrays in the context on
 * its first call; this call allocates nothing (no cudaMalloc, no library call
 * that allocates) and keeps them in one static device array of
 * ROMB_NOALLOC_SCRATCH_BYTES instead.  The problem must fit in it: with
 * C cells and control grid (m*nx+1) x (m*ny+1) = G points it needs
 *   8 * (C * (277 + 2 (m+1)^2) + 2 G + 64) bytes plus at most 7 * 255 of
 * alignment, e.g. 10.7 MB for 64 x 64 cells at m = 3 and roughly 5,800 cells
 * at m = 4; larger problems return ROMB_E_SCRATCH and change nothing.
 *
 * Set-up: every call, with the context's device current, looks up the
 * array's device address with cudaGetSymbolAddress (so a reset or re-created
 * device context never leaves a stale address behind).  The first call on a
 * device may load the library's device code and its static memory: make it
 * before any stream capture, at a point where that one-time load is
 * acceptable.  Every call clears the part of the array it uses before using
 * it, and synchronises the context's stream before it returns.
 *
 * The array is shared by every context on the device: calls that overlap in
 * time on one device (from several host threads, or from contexts on
 * unordered streams) race on it and must be serialised by the caller. */
romb_status romb_compliance_grad_noalloc(romb_ctx* ctx, double* compliance, double* dc_dctrl, double* dc_dR,
                                         double* dc_dmu);

/* FMA issue rate of this GPU (a measurement utility; the paper has no
 * counterpart): enqueues on `cuda_stream` (a cudaStream_t, NULL: the legacy
 * default stream) one kernel of `blocks` x `threads` threads (threads a
 * multiple of 32, at most 256), each running 8 independent chains of
 * 16 * iters dependent FMAs in FP64 (precision 0) or FP32 (precision 1).
 * `out` is device memory of blocks * threads elements of that type (written,
 * so the chains are kept); *flops receives the floating-point operations the
 * launch performs (2 per FMA).  The caller times the launch on its stream.
 * Errors: ROMB_E_ARG, ROMB_E_CUDA. */
romb_status romb_fma_probe(int precision, int blocks, int threads, int iters, void* cuda_stream, void* out,
                           double* flops);

/* How romb_bddc_solve forms the traction loads (Eq. ELA constitutive on the
 * conformal part of the loaded edges, Sec. 2.2.3):
 *   ROMB_LOADS_QUADRATURE (default): Gauss quadrature of j t b_s on the solid
 *     intervals of every loaded cell edge;
 *   ROMB_LOADS_REDUCED: the reduced model of the force integrals (Eq. SPEED
 *     L ext, reduced as in Sec. 4.2): J_e(mu) = U_f theta_f(mu) with theta_f
 *     interpolated like I_r (Algorithm 5), contracted with t_hat = j t at the
 *     q+1 GLL nodes of the edge.  Needs cell matrices from romb_assemble and
 *     models of file version 2 (else a solve returns ROMB_E_STATE before
 *     enqueuing any work).
 * The choice stays with the context.  Errors: ROMB_E_ARG. */
enum { ROMB_LOADS_QUADRATURE = 0, ROMB_LOADS_REDUCED = 1 };
romb_status romb_set_load_form(romb_ctx* ctx, int form);

/* Precision in which the BDDC preconditioner (Algorithm 1) is applied: its
 * fine operator D F D, the restriction and prolongation Phi and the coarse
 * substitutions with the factor of S_C.  ROMB_PRECOND_AUTO (default): FP32
 * after a split-precision assembly, FP64 otherwise; ROMB_PRECOND_FP64 /
 * ROMB_PRECOND_FP32 force one.  The factorisations, the operator S, the PCG
 * vectors, dot products and the stopping test stay FP64 in every case: the
 * iterate converges to the same solution and only the preconditioner (an
 * SPD operator up to FP32 rounding) changes.  Takes effect at the next
 * romb_factor.  Errors: ROMB_E_ARG for another value. */
enum { ROMB_PRECOND_AUTO = -1, ROMB_PRECOND_FP64 = 0, ROMB_PRECOND_FP32 = 1 };
romb_status romb_set_precond_precision(romb_ctx* ctx, int mode);

/* A constant body force (bx, by) per unit physical area on the solid part of
 * every cell (the volume term of Eq. SPEED L ext): with b_hat = det J b at the
 * (q+1)^2 interpolation nodes (Eq. FAST b interpolation) and the reduced
 * volume integrals V[k][k3] = int over the trimmed cell of B_k L_k3, node k
 * carries sum_k3 V[k][k3] b_hat(xi_k3).  The interior loads are condensed on
 * the skeleton and enter the recovery (Sec. 3.2).  Needs ROMB_LOADS_REDUCED
 * and force models trained with a volume part (romb_train_spec.body; else a
 * solve returns ROMB_E_STATE before enqueuing any work); (0, 0) switches it
 * off.  The compliance gradient covers the quadrature traction loads only
 * and returns ROMB_E_STATE after a solve with body forces or reduced loads.
 * The setting stays with the context.  Errors: ROMB_E_ARG (non-finite). */
romb_status romb_set_body_force(romb_ctx* ctx, double bx, double by);

/* Phase timings (ms, CUDA events) of the last calls: [0] theta, Chat and the
 * coarse DoFs' edge functionals, [1] contraction,
 * [2] local factor, [3] coarse assembly + factor, [4] PCG, [5] recovery,
 * [6] host<->device copies, [7] total.  flags_out: [ncells] per-cell bits
 * (1 out of box, 2 bad map, 4 not SPD, 8 non-finite, 16 assembled by the
 * exact fallback of romb_set_exact_fallback); either may be NULL. */
romb_status romb_stats(romb_ctx* ctx, double* phase_ms, int* flags_out);

/* Fallback for cells whose reduced-model stiffness is not positive definite
 * (the MDEIM error of a nearly void cell can exceed the alpha-stabilisation
 * rho I_Pi; Sec. 5.1.2 asks to retrain such models).  On (default), when
 * romb_factor meets a non-positive pivot in at most max_cells cells of a
 * reduced-model assembly, it integrates those cells' tensors I(mu) exactly
 * (the trimmed quadrature of the GPU trainer), forms their K by Algorithm 4
 * in FP64 (theta of the cell set to (rho, 1 - rho) against [I_Pi; I(mu)]),
 * marks them with flag 16 and factorises again; a second failure returns
 * ROMB_E_NOT_SPD.  Off (max_cells = 0): the failure is returned at once.
 * The exact tensors are kept per context and (family, mu), so a cell met
 * again skips the quadrature (one snapshot takes ~0.3 s on one CTA).
 * Errors: ROMB_E_ARG (max_cells < 0). */
romb_status romb_set_exact_fallback(romb_ctx* ctx, int max_cells);

/* Number of CUDA kernels this context has launched since romb_create. */
long long romb_launch_count(romb_ctx* ctx);

/* Copy an internal per-cell array to host memory (inspection and testing).
 * `bytes` must equal the field's size; see romb_field_bytes. */
typedef enum {
  ROMB_FIELD_CHAT = 0,     /* [cells][(q+1)^2][2][2][2][2] f64: C_{i1 j1 i2 j2 k}     */
  ROMB_FIELD_THETA = 1,    /* [cells][n_r+1] f64: (rho, (1-rho) I_r(mu))            */
  ROMB_FIELD_K = 2,        /* [cells][ndof(ndof+1)/2] f64: K, packed upper, row-major */
  ROMB_FIELD_S = 3,        /* [cells][nU*(nU+1)/2] f64: Schur complement, packed     */
  ROMB_FIELD_PSI = 4,      /* [cells][nU][20] f64: coarse basis (absent slots zero)  */
  ROMB_FIELD_SC_LOCAL = 5, /* [cells][20][20] f64: Psi^T S Psi                       */
  ROMB_FIELD_D = 6,        /* [cells][nU] f64: partition of unity                    */
  ROMB_FIELD_FINE = 7,     /* [cells][nU*(nU+1)/2] f64: D F D, packed                */
  ROMB_FIELD_FLAGS = 8,    /* [cells] int32                                          */
  ROMB_FIELD_LOADS = 9     /* [cells][nU] f64: traction loads of the first set of the
                              last romb_bddc_solve on the skeleton slots            */
} romb_field;
size_t romb_field_bytes(romb_ctx* ctx, int field);
romb_status romb_read(romb_ctx* ctx, int field, void* out, size_t bytes);

/* Offline ROM training (Sec. 4.2 and the offline phase of Sec. 4.4), on the
 * host CPU: snapshots I(mu_s) of Eq. (MDEIM I) at the given threshold samples
 * (e.g. a Latin hypercube in [lo,hi]^4), the leading n_r left singular vectors,
 * the magic points of Algorithm 3 and the I_r samples on the (r+1)^4 tensor
 * GLL grid of the box; written as a ROM file (format above).  samples:
 * [n_s][4] host array; n_threads host threads (0: all cores).
 * Errors: ROMB_E_ARG (bad spec, n_r > n_s, unwritable path), ROMB_E_NAN. */
typedef struct {
  int family;     /* 0 circle hole, 1 cross, 2..5 TPMS (Table GEO tpms) */
  int basis;      /* 0 GLL Lagrange, 1 Bernstein              */
  int p, q, r;    /* cell degree (3..8), q = 2, grid degree r */
  int n_r;        /* reduced basis size                       */
  int n_threads;
  double lo, hi;  /* parameter box [lo, hi]^4                 */
  int body;       /* nonzero: the force model also reduces the volume integrals of
                     body forces (Eq. SPEED L ext, romb_set_body_force)            */
} romb_train_spec;
romb_status romb_train(const romb_train_spec* spec, const double* samples, int n_s, const char* rom_path);

/* The same training on the GPU `device`: the snapshot moments and
 * snapshots (one CTA per parameter point, the adaptive panel quadrature of
 * the host trainer), the snapshot Gram matrix and U_r (FP64 GEMM kernels;
 * the n_s x n_s eigenvectors on the host), U_r orthonormalised by two passes
 * of Cholesky QR, the magic points of Algorithm 3 (residual and arg-max on
 * the device, ties to the lowest index) and the I_r samples on the
 * (r+1)^4 grid (moments and magic-point entries on the device).  Same file
 * format; spec->n_threads is ignored.  Allocates and frees its own device
 * memory.  Errors: ROMB_E_ARG, ROMB_E_NAN, ROMB_E_CUDA. */
romb_status romb_train_gpu(int device, const romb_train_spec* spec, const double* samples, int n_s,
                           const char* rom_path);

/* Clustered training (Sec. 4.2.1): the box [lo, hi]^4 is split into n_k
 * equal subintervals per threshold (n_k = 1 or 2), cluster
 * k = k1 + n_k (k2 + n_k (k3 + n_k k4)) with k_d the subinterval of mu_d, and
 * each cluster is trained as romb_train_gpu trains one box, on its own
 * samples and its own (r+1)^4 GLL grid.  samples: [n_k^4][n_s][4] host array,
 * block k drawn in cluster k's box.  One file with n_k in its header and the
 * clusters' sections in cluster order (format above).  Errors as
 * romb_train_gpu. */
romb_status romb_train_gpu_clustered(int device, const romb_train_spec* spec, int n_k, const double* samples,
                                     int n_s, const char* rom_path);

/* Snapshots I(mu_k) (Eq. MDEIM I) of n threshold points mu [n][4] (host) by
 * the GPU trainer's quadrature: I_out [n][n_i] host array. */
romb_status romb_train_snapshots_gpu(int device, const romb_train_spec* spec, const double* mu, int n,
                                     double* I_out);

/* One fast-assembly snapshot I(mu) (Eq. MDEIM I) by the trainer's quadrature:
 * I_out[n_i], n_i = (p+1)^4 (q+1)^2 4, layout as in the ROM file. */
romb_status romb_train_snapshot(const romb_train_spec* spec, const double* mu4, double* I_out);

#ifdef __cplusplus
}
#endif
#endif /* ROMB_H */
