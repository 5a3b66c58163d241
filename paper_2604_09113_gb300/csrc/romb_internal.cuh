// Internal declarations of the romb library (context, device buffers, kernel
// launchers).  Everything here is private to the shared library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <map>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/romb.h"

#define ROMB_MAX_FAMILIES 8
#define ROMB_MAX_MODELS 64   // resident reduced models: one per (family, cluster)
#define ROMB_MAX_NK 2        // clusters per threshold parameter (n_k^4 models per family)
#define ROMB_MAX_IV 4        // solid intervals of one trimmed line, at most (trim.cuh)
#define ROMB_MAX_P 8
#define ROMB_NSLOT 20      // local coarse slots: 4 corners x 2 + 4 edges x 3

// Per-cell error bits (romb_stats flags).
#define ROMB_FLAG_OUT_OF_BOX 1
#define ROMB_FLAG_BAD_MAP 2
#define ROMB_FLAG_NOT_SPD 4
#define ROMB_FLAG_NAN 8
#define ROMB_FLAG_EXACT 16   // K of the cell from the exact tensor (romb_set_exact_fallback)

#define ROMB_CUDA(call)                                                     \
  do {                                                                      \
    cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess) {                                                \
      romb_set_error(std::string(#call) + ": " + cudaGetErrorString(e_));   \
      return ROMB_E_CUDA;                                                   \
    }                                                                       \
  } while (0)

void romb_set_error(const std::string& s);

// One loaded reduced model (Sec. 4.2) of one family and one cluster (Sec.
// 4.2.1), resident in HBM.  Its box is [lo4[d], hi4[d]] per threshold.
struct RombRom {
  bool loaded = false;
  int family = -1, kind = 0, p = 0, q = 0, r = 0, n_r = 0, cluster = 0;
  double lo4[4] = {0, 0, 0, 0}, hi4[4] = {0, 0, 0, 0};
  long long n_half = 0;        // pairs k1 <= k2 times 4 (q+1)^2 columns
  double* U64 = nullptr;       // [(n_r+1)][n_half]: row 0 = I_Pi, rows 1.. = U_r
  float* Utiles = nullptr;     // tensor-core operand: N-tiles of 144 columns, TF32 hi then lo, canonical layout
  uint16_t* Utiles16 = nullptr;   // the same tiles with BF16 hi / lo (16-bit canonical layout)
  int ntiles = 0;
  int kpad16 = 0;              // n_r+1 rounded up to the BF16 MMA K step (16)
  double* A = nullptr;         // [n_r][(r+1)^4]
  double* At = nullptr;        // [(r+1)^4][n_r]
  float2* At2 = nullptr;       // the same as (hi, lo) FP32 pairs, hi + lo = At to ~48 bits (double-float theta)
  int kpad = 0;                // n_r+1 rounded up for the tensor-core K dimension
  // reduced model of the force integrals J(mu) (file version 2; absent: null)
  int force_nf = 0, force_rf = 0;
  double* force_U = nullptr;   // [r_f][n_f], n_f = 4 (p+1) (q+1): J[e][s][k]
  double* force_At = nullptr;  // [(r+1)^4][r_f]
};

// The models of one family: slots [slot0, slot0 + n_k^4), cluster
// k = k1 + n_k (k2 + n_k (k3 + n_k k4)) on the box [lo, hi]^4 (n_k = 0: none).
struct RombCtxFamilies {
  int n_k = 0, slot0 = -1;
  double lo = 0, hi = 0;
};

// Nested-dissection coarse solver (a5): symbolic tree built on the host from
// the lattice shape, numeric fronts on the device.
struct NdFront {
  int ns = 0, nb = 0;          // eliminated (separator) rows, update (boundary) rows
  long long off = 0;           // offset of the dense front (n x n, n = ns + nb) in the pool
  long long upd_off = 0;       // offset of its update matrix (nb x nb)
  int level = 0, parent = -1;
  long long idx_off = 0;       // offset of its n global coarse indices
  std::vector<int> children;
};

struct NdPlan {
  int n = 0;                   // coarse unknowns (Dirichlet ones excluded)
  std::vector<NdFront> fronts;
  std::vector<std::vector<int>> levels;   // front ids per level, leaves first
  long long pool = 0, upd_pool = 0, idx_total = 0;
  // device
  double* F = nullptr;         // dense fronts
  double* Upd = nullptr;       // update matrices
  int* idx = nullptr;          // global coarse index of each front row
  int* d_meta = nullptr;       // per-front {ns, nb, off_lo, off_hi, upd_lo, upd_hi, idx_lo, idx_hi}
  // child extend-add maps: for each child row, its position in the parent front
  int* d_cmap = nullptr;
  long long cmap_total = 0;
  std::vector<long long> cmap_off;        // per front (as child)
  // cell -> leaf assembly: for each cell its leaf and the leaf-row of each slot
  int* d_cell_leaf = nullptr;
  int* d_cell_pos = nullptr;              // [cells][20], -1 absent
  double* d_rhs = nullptr;                // [n] work vector
  double* d_ybuf = nullptr;               // per-front update buffers for solves
  long long ybuf_total = 0;
  std::vector<long long> ybuf_off;
  int* d_ybuf_off = nullptr;
  int* d_children = nullptr;              // flattened child lists
  int* d_child_off = nullptr;             // [nfronts+1]
  std::vector<int*> d_level_fronts;       // per level: device list of front ids
  int max_ns_small = 0;
};

// State of one PCG solve (Algorithm 1 inside CG) and its interior recovery:
// the streams it runs on, its skeleton vectors and cell-local scratch, the
// coarse-solve buffers and the captured iteration graph.  romb_bddc_solve
// runs several load sets at once on separate lanes; lane 0 runs on the
// context's stream and holds the state the compliance gradient reads.
#define ROMB_MAX_LANES 16
struct PcgLane {
  cudaStream_t stream = nullptr;   // main stream (lane 0: the context's stream)
  cudaStream_t side = nullptr;     // highest priority: coarse correction
  cudaEvent_t evfork = nullptr, evjoin = nullptr, ev0 = nullptr, ev1 = nullptr;
  bool have_streams = false, own_stream = false;
  double* h_red = nullptr;         // pinned: [0] r.r, [1] f.f, [3] iterations
  // lattice-dependent device buffers (freed with the lattice)
  bool have_bufs = false;
  double *d_f = nullptr, *d_x = nullptr, *d_r = nullptr, *d_z = nullptr, *d_pv = nullptr, *d_q = nullptr;
  double* d_red = nullptr;         // scalars and reduction partials
  double* d_fU = nullptr;          // [cells][nU] skeleton-slot forces
  double* d_cloc = nullptr;        // [cells][20] coarse restriction
  double* d_yloc = nullptr;        // [cells][nU] cell-local scratch
  double* d_coarse = nullptr;      // [2][ncoarse_all] coarse right-hand side and solution
  double* d_u = nullptr;           // nodal output [nodes][2]
  double* d_traction = nullptr;    // [4][2]
  unsigned char* d_forcetab = nullptr;   // reduced force models by slot (loads_rom_kernel)
  double* d_fI = nullptr;       // [cells][nI] interior body loads, then L^-1 f_I (recovery)
  bool body_on = false;         // this solve carries body forces
  double* nd_ybuf = nullptr;       // coarse-solve update vectors
  double* nd_sbuf = nullptr;       // coarse-solve forward results
  cudaGraphExec_t graph = nullptr; // the captured PCG loop (per factorisation)
  long long graph_launches = 0;
  bool device_loop = false;
  double nf = 0.0;                 // ||f|| of the lane's current load set
};

struct romb_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t budget = 0, used = 0, rom_bytes = 0;
  int sms = 0;
  std::vector<void*> allocs;       // lattice-dependent buffers
  std::vector<void*> rom_allocs;   // loaded reduced models
  std::unordered_map<void*, size_t> sizes;

  RombRom roms[ROMB_MAX_MODELS];   // by model slot
  RombCtxFamilies fams[ROMB_MAX_FAMILIES];
  int nslots = 0;

  // lattice
  bool have_lattice = false, assembled = false, factored = false;
  bool assembled_split = false;   // cell matrices from a split-precision form
  int nx = 0, ny = 0, p = 0, m = 0, basis = 0, ncells = 0, mem = 0;
  int nB = 0, ndof = 0, nI = 0, nU = 0, q = 2, nL = 9;
  long long kpack = 0, upack = 0;   // packed sizes of K and of nU x nU
  double E = 1, nu = 0.3, rho = 0;
  unsigned dmask = 0;
  double traction[8] = {0};
  int prec = 0;
  int load_form = 0;            // 0 direct edge quadrature, 1 reduced force model (romb_set_load_form)
  double body[2] = {0.0, 0.0};  // constant body force per unit area (romb_set_body_force)

  double* d_ctrl = nullptr;
  double* d_mu = nullptr;
  int32_t* d_family = nullptr;
  int32_t* d_flags = nullptr;

  // layout of the present cells (Sec. 5.2.2); cells are numbered 0..ncells-1
  // in increasing grid index c = cx + nx cy, and every per-cell array below
  // is in that order
  bool layout = false;               // cell_present or edge_clamped given
  std::vector<uint8_t> h_present;    // [nx*ny] as given (empty: every cell)
  std::vector<uint8_t> h_clamped;    // [nx*ny][4] as given (empty: none)
  std::vector<int> h_cell_grid;      // [ncells] grid index of each present cell
  int* d_cell_grid = nullptr;        // [ncells]
  int* d_grid_cell = nullptr;        // [nx*ny] present-cell number, -1 absent
  uint8_t* d_node_fixed = nullptr;   // [skeleton nodes] clamped or of no present cell
  double* d_stage = nullptr;         // [nx*ny][4] grid-indexed inputs on their way to d_mu

  // per-cell arrays
  double* d_chat = nullptr;     // [cells][nL][16]
  float* d_chat32 = nullptr;    // [cells][144] FP32 copy for the tensor-core epilogue
  double* d_theta = nullptr;    // [cells][kmax]
  float* d_theta_hi = nullptr;  // [cells][kpad] tensor-core operand (hi)
  float* d_theta_lo = nullptr;  // [cells][kpad] (lo)
  int32_t* d_slot = nullptr;    // [cells] model slot of each cell (FindCluster of its family)
  int* d_famlist = nullptr;     // cells grouped by model slot
  int2* d_pairs = nullptr;      // (k1, k2), k1 <= k2, in pair order
  int famcount[ROMB_MAX_MODELS] = {0};   // cells per model slot
  int famstart[ROMB_MAX_MODELS] = {0};
  double* d_K = nullptr;        // [cells][kpack]
  double* d_kdiag = nullptr;    // [cells][nU] diagonal of K at the skeleton slots
  double* d_ktot = nullptr;     // [skeleton DoFs] sum of the diagonals of sharing cells
  double* d_LII = nullptr;      // [cells][nI(nI+1)/2] Cholesky factor of K_II, packed lower
  double* d_W = nullptr;        // [cells][nI][nU]  L_II^-1 K_IU
  double* d_S = nullptr;        // [cells][upack]
  double* d_G = nullptr;        // [cells][upack]   D F D
  double* d_Phi = nullptr;      // [cells][nU][20]  D Psi
  double* d_Psi = nullptr;      // [cells][nU][20]
  double* d_SCl = nullptr;      // [cells][20][20]
  double* d_D = nullptr;        // [cells][nU]
  double* d_efun = nullptr;     // [cells][4][p+1][3] edge functionals (a, m1, m2) of the coarse DoFs
  bool efun_ready = false;      // d_efun holds this lattice's functionals
  double* d_eiv = nullptr;      // [cells][4][1 + 2 ROMB_MAX_IV] solid intervals of each cell edge

  // skeleton
  long long nskel_nodes = 0, nskel = 0;   // nodes / DoFs (Dirichlet ones included, masked)
  int* d_ucell_map = nullptr;   // [cells][nU] skeleton DoF of each local U slot (-1 Dirichlet)
  int* d_islot = nullptr;       // [nI] local DoF of each interior slot (device table)
  int* d_uslot = nullptr;       // [nU] local DoF of each skeleton slot

  // coarse
  long long ncoarse_all = 0;    // all coarse DoFs incl. Dirichlet (masked)
  int* d_cmap = nullptr;        // [cells][20] global coarse DoF (-1 absent)
  int* d_cnum = nullptr;        // [ncoarse_all] -> ND unknown (-1 Dirichlet)
  NdPlan nd;

  // reduction scratch of the assembly, the factor checks and the compliance
  double* d_red = nullptr;
  double* h_red = nullptr;      // pinned host copy
  int* d_pcg_err = nullptr;     // set by a PCG cell kernel whose staging copy timed out
  int ca_grid[4] = {0, 0, 0, 0};   // persistent grid of the cell operator kernels per mode (+1: FP32)
  // split-precision forms: the preconditioner's operators D F D and Phi (and
  // the coarse solve's B) in FP32, set by romb_factor
  bool pre32 = false;
  int precond_mode = -1;        // romb_set_precond_precision (survives a new lattice)
  int fallback_max = 64;        // romb_set_exact_fallback (survives a new lattice)
  // exact tensors of the fallback, row 1 of U' in the half layout, keyed by
  // (family, basis, p, q, mu): a cell met again skips the quadrature
  std::map<std::vector<double>, std::vector<double>> exact_cache;
  float* d_G32 = nullptr;       // [cells][nU][nU]
  float* d_Phi32 = nullptr;     // [cells][nU][20]
  int* d_cowner = nullptr;      // [ncoarse_all][4] cell*20 + slot of each owner (-1 none)
  PcgLane lane[ROMB_MAX_LANES]; // PCG solves (see PcgLane)

  // gradient
  bool solved = false, assembled_rom = false;
  double* d_gW = nullptr;       // [cells][144] sum_{k1 k2} u u I'
  double* d_gQ = nullptr;       // [cells][128] u^T dK/dtheta_t u
  double* d_gloc = nullptr;     // [cells][(m+1)^2][2] local control-point gradient
  double* d_gdmu = nullptr;     // [cells][4]
  double* d_gdctrl = nullptr;   // [ctrl][2]

  // timing and launch accounting
  long long launches = 0;      // kernels launched by this context so far
  cudaEvent_t ev[16];
  double phase_ms[8] = {0};
};

// allocation helpers (respect the budget)
romb_status romb_alloc(romb_ctx* c, void** p, size_t bytes);
romb_status romb_alloc_persist(romb_ctx* c, void** p, size_t bytes);
void romb_free_lattice(romb_ctx* c);
template <class T>
inline romb_status romb_alloc_t(romb_ctx* c, T** p, size_t n) {
  return romb_alloc(c, (void**)p, n * sizeof(T));
}
void romb_free_all(romb_ctx* c);

// kernel launchers (each returns ROMB_OK or ROMB_E_CUDA)
romb_status launch_theta(romb_ctx* c);
romb_status launch_edge_functionals(romb_ctx* c);
romb_status launch_assemble_cells_fp64(romb_ctx* c, const double* U, long long n_half, int K,
                                      const int* d_list, int count);
romb_status launch_assemble_fp64(romb_ctx* c);
romb_status launch_assemble_tc(romb_ctx* c);
romb_status launch_factor(romb_ctx* c);
romb_status coarse_build(romb_ctx* c);      // symbolic (once per lattice shape)
romb_status coarse_factor(romb_ctx* c);     // numeric
romb_status coarse_solve(romb_ctx* c, const double* d_in, double* d_out, cudaStream_t st, double* ybuf,
                         double* sbuf);
romb_status coarse_lane_buffers(romb_ctx* c, double** ybuf, double** sbuf);   // sized like lane 0's
romb_status coarse_solve_check(romb_ctx* c);   // staging timeouts of the solve kernels
romb_status launch_ktot(romb_ctx* c);
romb_status launch_flag_or(romb_ctx* c, int* d_any);
romb_status launch_grad(romb_ctx* c, double* d_dctrl, double* d_dmu);
romb_status launch_grad_scratch(romb_ctx* c, double* W, double* Q, double* gloc, double* d_dctrl, double* d_dmu);
romb_status romb_dot(romb_ctx* c, const double* a, const double* b, long long n, double* out);
romb_status launch_pack_dense(romb_ctx* c, const double* d_dense);
// A PCG solve on lane L in two halves: pcg_begin enqueues the loads and
// ||f||^2 (read by the host after a stream synchronisation); pcg_finish
// enqueues the PCG loop, the recovery into L.d_u and the copy of the
// iteration count and residual to L.h_red; pcg_result reads them after the
// lane's stream has been synchronised.
romb_status pcg_begin(romb_ctx* c, PcgLane& L, const double* traction_dev_or_host, bool traction_on_device);
romb_status pcg_finish(romb_ctx* c, PcgLane& L, double rtol, int maxit);
romb_status pcg_result(romb_ctx* c, PcgLane& L, double rtol, int maxit, int* iters, double* relres);
romb_status pcg_lane_streams(romb_ctx* c, PcgLane& L, bool main_is_context_stream);
void pcg_lane_destroy(PcgLane& L);

// reduced model of the force integrals J(mu) (train.cu; file format version 2)
struct RombForceModel {
  int n_f = 0, r_f = 0;
  std::vector<double> U;          // [r_f][n_f]
  std::vector<double> A;          // [r_f][(r+1)^4]
  std::vector<long long> magic;   // [r_f]
};
romb_status train_force_model(const romb_train_spec* sp, const double* samples, int n_s, RombForceModel* out);
// The same on the box [lo4[d], hi4[d]] per threshold (one cluster).
romb_status train_force_model_box(const romb_train_spec* sp, const double* lo4, const double* hi4,
                                  const double* samples, int n_s, RombForceModel* out);
bool write_force_section(FILE* f, const RombForceModel& m);

// host-trainer pieces the GPU trainer reuses (train.cu)
romb_status train_host_tables(const romb_train_spec* sp, std::vector<double>& F, int* D, int* nF,
                              std::vector<double>& gx, std::vector<double>& gw, std::vector<double>& Ipi);
void train_jacobi_eig(int n, std::vector<double>& A, std::vector<double>& w, std::vector<double>& V);

void tc_tile_rom(const std::vector<double>& U, long long n_half, int K, int kpad, std::vector<float>& tiles,
                 int* ntiles);
void tc_tile_rom_bf16(const std::vector<double>& U, long long n_half, int K, int kpad, std::vector<uint16_t>& tiles);

// small host helpers
inline long long tri(long long n) { return n * (n + 1) / 2; }
