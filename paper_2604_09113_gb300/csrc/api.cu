// C-ABI entry points of romb: context, memory, ROM loading, lattice set-up and
// the orchestration of the online phase (Sec. 4.4): assemble -> factor -> solve.
#include <math.h>
#include <cmath>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "romb_internal.cuh"
#include "tables.cuh"

static thread_local std::string g_err;
void romb_set_error(const std::string& s) { g_err = s; }

extern "C" const char* romb_strerror(romb_status s) {
  switch (s) {
    case ROMB_OK: return "ok";
    case ROMB_E_ARG: return "invalid argument";
    case ROMB_E_CUDA: return g_err.empty() ? "CUDA error" : g_err.c_str();
    case ROMB_E_OOM: return "out of device memory or budget";
    case ROMB_E_OUT_OF_BOX: return "threshold outside the trained ROM box";
    case ROMB_E_BAD_MAP: return "non-positive Jacobian determinant at an interpolation node";
    case ROMB_E_NOT_SPD: return "non-positive pivot in a Cholesky factorisation";
    case ROMB_E_NOT_CONVERGED: return "PCG did not converge within maxit";
    case ROMB_E_NAN: return "non-finite value";
    case ROMB_E_FORMAT: return "malformed ROM file";
    case ROMB_E_STATE: return "call out of order";
    case ROMB_E_SCRATCH: return "problem larger than the fixed scratch of the no-allocation call";
  }
  return "unknown status";
}

static romb_status alloc_into(romb_ctx* c, void** p, size_t bytes, std::vector<void*>& list) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  if (c->budget && c->used + bytes > c->budget) return ROMB_E_OOM;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    *p = nullptr;
    return ROMB_E_OOM;
  }
  c->used += bytes;
  c->sizes[*p] = bytes;
  if (&list == &c->rom_allocs) c->rom_bytes += bytes;
  list.push_back(*p);
  return ROMB_OK;
}

romb_status romb_alloc(romb_ctx* c, void** p, size_t bytes) { return alloc_into(c, p, bytes, c->allocs); }
romb_status romb_alloc_persist(romb_ctx* c, void** p, size_t bytes) {
  return alloc_into(c, p, bytes, c->rom_allocs);
}

static void romb_free_ptr(romb_ctx* c, void* p) {
  if (!p) return;
  for (auto* list : {&c->allocs, &c->rom_allocs}) {
    auto it = std::find(list->begin(), list->end(), p);
    if (it != list->end()) {
      if (list == &c->rom_allocs) c->rom_bytes -= c->sizes[p];
      list->erase(it);
    }
  }
  c->used -= c->sizes[p];
  c->sizes.erase(p);
  cudaFree(p);
}

// Free every lattice-dependent buffer (the loaded ROMs stay).
void romb_free_lattice(romb_ctx* c) {
  for (PcgLane& L : c->lane)
    if (L.graph) {
      cudaGraphExecDestroy(L.graph);
      L.graph = nullptr;
    }
  for (void* p : c->allocs) {
    cudaFree(p);
    c->sizes.erase(p);
  }
  c->allocs.clear();
  auto sizes = c->sizes;
  const size_t rom_bytes = c->rom_bytes;
  std::vector<RombRom> roms(c->roms, c->roms + ROMB_MAX_MODELS);
  RombCtxFamilies fams[ROMB_MAX_FAMILIES];
  for (int i = 0; i < ROMB_MAX_FAMILIES; ++i) fams[i] = c->fams[i];
  const int nslots = c->nslots;
  std::vector<void*> keep = c->rom_allocs;
  cudaStream_t st = c->stream;
  bool own = c->own_stream;
  int dev = c->device, sms = c->sms;
  size_t budget = c->budget;
  double* h_red = c->h_red;
  cudaEvent_t ev[16];
  for (int i = 0; i < 16; ++i) ev[i] = c->ev[i];
  // lanes keep their streams, events and pinned words; their device buffers
  // went with the lattice
  const int load_form = c->load_form, precond_mode = c->precond_mode, fallback_max = c->fallback_max;
  const double body[2] = {c->body[0], c->body[1]};
  PcgLane lanes[ROMB_MAX_LANES];
  for (int k = 0; k < ROMB_MAX_LANES; ++k) {
    const PcgLane& o = c->lane[k];
    PcgLane& L = lanes[k];
    L.stream = o.stream;
    L.side = o.side;
    L.evfork = o.evfork;
    L.evjoin = o.evjoin;
    L.ev0 = o.ev0;
    L.ev1 = o.ev1;
    L.have_streams = o.have_streams;
    L.own_stream = o.own_stream;
    L.h_red = o.h_red;
  }
  *c = romb_ctx();
  for (int k = 0; k < ROMB_MAX_LANES; ++k) c->lane[k] = lanes[k];
  c->load_form = load_form;
  c->precond_mode = precond_mode;
  c->fallback_max = fallback_max;
  c->body[0] = body[0];
  c->body[1] = body[1];
  for (int i = 0; i < ROMB_MAX_MODELS; ++i) c->roms[i] = roms[i];
  for (int i = 0; i < ROMB_MAX_FAMILIES; ++i) c->fams[i] = fams[i];
  c->nslots = nslots;
  c->rom_allocs = keep;
  c->stream = st;
  c->own_stream = own;
  c->device = dev;
  c->sms = sms;
  c->budget = budget;
  c->h_red = h_red;
  for (int i = 0; i < 16; ++i) c->ev[i] = ev[i];
  c->sizes = sizes;
  c->rom_bytes = rom_bytes;
  c->used = rom_bytes;
}

void romb_free_all(romb_ctx* c) {
  for (void* p : c->allocs) cudaFree(p);
  for (void* p : c->rom_allocs) cudaFree(p);
  c->allocs.clear();
  c->rom_allocs.clear();
  c->used = 0;
}

extern "C" romb_status romb_create(romb_ctx** out, int device, size_t budget, void* stream) {
  if (!out) return ROMB_E_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    (void)cudaGetLastError();
    romb_set_error("no CUDA device");
    return ROMB_E_CUDA;
  }
  ROMB_CUDA(cudaSetDevice(device));
  romb_ctx* c = new romb_ctx();
  c->device = device;
  c->budget = budget;
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
  if (stream) {
    c->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return ROMB_E_CUDA;
    }
    c->own_stream = true;
  }
  for (auto& e : c->ev) cudaEventCreate(&e);
  if (pcg_lane_streams(c, c->lane[0], true) != ROMB_OK) {
    (void)cudaGetLastError();
    romb_set_error("romb_create: stream or event creation failed");
    pcg_lane_destroy(c->lane[0]);
    delete c;
    return ROMB_E_CUDA;
  }
  if (cudaMallocHost(&c->h_red, 64 * sizeof(double)) != cudaSuccess) {
    delete c;
    return ROMB_E_OOM;
  }
  *out = c;
  return ROMB_OK;
}

extern "C" void romb_destroy(romb_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  for (PcgLane& L : c->lane) {
    if (L.have_streams && L.own_stream) cudaStreamSynchronize(L.stream);
    pcg_lane_destroy(L);
  }
  romb_free_all(c);
  for (int l = 0; l < (int)c->nd.d_level_fronts.size(); ++l) c->nd.d_level_fronts[l] = nullptr;
  for (auto& e : c->ev) cudaEventDestroy(e);
  if (c->h_red) cudaFreeHost(c->h_red);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}

// ---------------------------------------------------------------------------
// ROM loading
// ---------------------------------------------------------------------------
static bool rd(FILE* f, void* p, size_t n) { return fread(p, 1, n, f) == n; }

// Release the device arrays of one model slot.
static void free_model(romb_ctx* c, RombRom& R) {
  if (R.loaded) {
    romb_free_ptr(c, R.U64);
    romb_free_ptr(c, R.Utiles);
    romb_free_ptr(c, R.Utiles16);
    romb_free_ptr(c, R.A);
    romb_free_ptr(c, R.At);
    romb_free_ptr(c, R.At2);
    romb_free_ptr(c, R.force_U);
    romb_free_ptr(c, R.force_At);
  }
  R = RombRom();
}

// Convert one cluster's model to the device layouts and install it in R.
static romb_status install_model(romb_ctx* c, RombRom& R, int family, int kind, int p, int q, int r, int n_r,
                                 long long n_i, long long ngrid, const std::vector<double>& Ipi,
                                 const std::vector<double>& U, const std::vector<double>& A,
                                 const std::vector<double>& Uf, const std::vector<double>& Af, const int64_t* fhdr) {
  const int nB = (p + 1) * (p + 1), nL = (q + 1) * (q + 1);
  // Rearrange into the pair-major half layout used by the contraction: row t of
  // U' is I_Pi (t = 0) or U_r column t-1; column (pair(k1<=k2), k3, j1, j2).
  const long long npairs = (long long)nB * (nB + 1) / 2;
  const long long n_half = npairs * nL * 4;
  const int K = n_r + 1;
  std::vector<double> Uh((size_t)K * n_half);
  long long pr = 0;
  for (int k1 = 0; k1 < nB; ++k1)
    for (int k2 = k1; k2 < nB; ++k2, ++pr)
      for (int e = 0; e < nL * 4; ++e) {
        const long long src = ((long long)k1 * nB + k2) * nL * 4 + e;
        const long long dst = pr * nL * 4 + e;
        Uh[dst] = Ipi[src];
        for (int t = 0; t < n_r; ++t) Uh[(size_t)(t + 1) * n_half + dst] = U[(size_t)t * n_i + src];
      }

  free_model(c, R);
  romb_status s;
  if (!Uf.empty()) {   // force model: U_f [r_f][n_f] and A_f transposed [grid][r_f]
    R.force_nf = (int)fhdr[0];
    R.force_rf = (int)fhdr[1];
    std::vector<double> Aft(Af.size());
    for (long long g = 0; g < ngrid; ++g)
      for (int t = 0; t < R.force_rf; ++t) Aft[(size_t)g * R.force_rf + t] = Af[(size_t)t * ngrid + g];
    if ((s = romb_alloc_persist(c, (void**)&R.force_U, 8 * Uf.size())) != ROMB_OK) return s;
    if ((s = romb_alloc_persist(c, (void**)&R.force_At, 8 * Aft.size())) != ROMB_OK) return s;
    ROMB_CUDA(cudaMemcpy(R.force_U, Uf.data(), 8 * Uf.size(), cudaMemcpyHostToDevice));
    ROMB_CUDA(cudaMemcpy(R.force_At, Aft.data(), 8 * Aft.size(), cudaMemcpyHostToDevice));
  }
  if ((s = romb_alloc_persist(c, (void**)&R.U64, 8 * Uh.size())) != ROMB_OK) return s;
  if ((s = romb_alloc_persist(c, (void**)&R.A, 8 * A.size())) != ROMB_OK) return s;
  if ((s = romb_alloc_persist(c, (void**)&R.At, 8 * A.size())) != ROMB_OK) return s;
  ROMB_CUDA(cudaMemcpy(R.U64, Uh.data(), 8 * Uh.size(), cudaMemcpyHostToDevice));
  ROMB_CUDA(cudaMemcpy(R.A, A.data(), 8 * A.size(), cudaMemcpyHostToDevice));
  {
    std::vector<double> At(A.size());
    for (long long g = 0; g < ngrid; ++g)
      for (int t = 0; t < n_r; ++t) At[(size_t)g * n_r + t] = A[(size_t)t * ngrid + g];
    ROMB_CUDA(cudaMemcpy(R.At, At.data(), 8 * At.size(), cudaMemcpyHostToDevice));
    std::vector<float2> At2(At.size());
    for (size_t i = 0; i < At.size(); ++i) {
      const float h = (float)At[i];
      At2[i] = make_float2(h, (float)(At[i] - (double)h));
    }
    if ((s = romb_alloc_persist(c, (void**)&R.At2, sizeof(float2) * At2.size())) != ROMB_OK) return s;
    ROMB_CUDA(cudaMemcpy(R.At2, At2.data(), sizeof(float2) * At2.size(), cudaMemcpyHostToDevice));
  }
  R.kpad = (K + 7) / 8 * 8;
  {
    // tensor-core operand tiles (TF32 hi/lo of rows 2.., rows 0-1 in FP64)
    std::vector<float> tiles;
    tc_tile_rom(Uh, n_half, K, R.kpad, tiles, &R.ntiles);
    if ((s = romb_alloc_persist(c, (void**)&R.Utiles, 4 * tiles.size())) != ROMB_OK) return s;
    ROMB_CUDA(cudaMemcpy(R.Utiles, tiles.data(), 4 * tiles.size(), cudaMemcpyHostToDevice));
    // and the BF16 hi / lo tiles of the same rows
    R.kpad16 = (K + 15) / 16 * 16;
    std::vector<uint16_t> t16;
    tc_tile_rom_bf16(Uh, n_half, K, R.kpad16, t16);
    if ((s = romb_alloc_persist(c, (void**)&R.Utiles16, 2 * t16.size())) != ROMB_OK) return s;
    ROMB_CUDA(cudaMemcpy(R.Utiles16, t16.data(), 2 * t16.size(), cudaMemcpyHostToDevice));
  }
  R.loaded = true;
  R.family = family;
  R.kind = kind;
  R.p = p;
  R.q = q;
  R.r = r;
  R.n_r = n_r;
  R.n_half = n_half;
  return ROMB_OK;
}

extern "C" romb_status romb_train_load(romb_ctx* c, const char* path, int* family_out) {
  if (!c || !path) return ROMB_E_ARG;
  ROMB_CUDA(cudaSetDevice(c->device));
  FILE* f = fopen(path, "rb");
  if (!f) return ROMB_E_ARG;
  unsigned char hdr[128];
  if (!rd(f, hdr, 128) || memcmp(hdr, "ROMBDDC1", 8) != 0) {
    fclose(f);
    return ROMB_E_FORMAT;
  }
  int32_t iv[8];
  double lohi[2];
  int64_t n_i;
  memcpy(iv, hdr + 8, 32);
  memcpy(lohi, hdr + 40, 16);
  memcpy(&n_i, hdr + 56, 8);
  const int version = iv[0], family = iv[1], kind = iv[2], p = iv[3], q = iv[4], r = iv[5], n_r = iv[6],
            n_k = iv[7];
  const int nB = (p + 1) * (p + 1), nL = (q + 1) * (q + 1);
  if ((version != 1 && version != 2) || n_k < 1 || n_k > ROMB_MAX_NK || family < 0 || family >= ROMB_MAX_FAMILIES || p < 3 || p > ROMB_MAX_P ||
      q != 2 || r < 1 || r > 10 || n_r < 1 || n_r > 127 || n_i != (int64_t)nB * nB * nL * 4 ||
      !(lohi[1] > lohi[0])) {
    fclose(f);
    return ROMB_E_FORMAT;
  }
  long long ngrid = 1;
  for (int d = 0; d < 4; ++d) ngrid *= (r + 1);
  int nK = 1;
  for (int d = 0; d < 4; ++d) nK *= n_k;
  std::vector<double> Ipi(n_i);
  if (!rd(f, Ipi.data(), 8 * n_i)) {
    fclose(f);
    return ROMB_E_FORMAT;
  }
  // model slots of the family: reused when the cluster count is unchanged
  RombCtxFamilies& F = c->fams[family];
  for (int k = 0; k < F.n_k * F.n_k * F.n_k * F.n_k; ++k) free_model(c, c->roms[F.slot0 + k]);
  if (F.n_k != n_k) {
    if (c->nslots + nK > ROMB_MAX_MODELS) {
      F = RombCtxFamilies();
      fclose(f);
      romb_set_error("romb_train_load: more than 64 resident models");
      return ROMB_E_ARG;
    }
    F.slot0 = c->nslots;
    c->nslots += nK;
  }
  F.n_k = 0;   // not usable until every cluster is in
  const double h = (lohi[1] - lohi[0]) / n_k;
  std::vector<double> U((size_t)n_r * n_i), A((size_t)n_r * ngrid), Uf, Af;
  std::vector<int64_t> magic(n_r);
  for (int k = 0; k < nK; ++k) {
    bool ok = rd(f, U.data(), 8 * U.size()) && rd(f, A.data(), 8 * A.size()) && rd(f, magic.data(), 8 * magic.size());
    // version 2: the reduced model of the force integrals J(mu) follows the magic points
    int64_t fhdr[2] = {0, 0};
    Uf.clear();
    Af.clear();
    if (ok && version == 2) {
      const long long ne = 4LL * (p + 1) * (q + 1), nv = (long long)nB * nL;
      ok = rd(f, fhdr, 16) && (fhdr[0] == ne || fhdr[0] == ne + nv) && fhdr[1] >= 1 && fhdr[1] <= fhdr[0] &&
           fhdr[1] <= 128;
      if (ok) {
        Uf.resize((size_t)fhdr[1] * fhdr[0]);
        Af.resize((size_t)fhdr[1] * ngrid);
        std::vector<int64_t> mf(fhdr[1]);
        ok = rd(f, Uf.data(), 8 * Uf.size()) && rd(f, Af.data(), 8 * Af.size()) && rd(f, mf.data(), 8 * mf.size());
      }
    }
    romb_status s = ok ? install_model(c, c->roms[F.slot0 + k], family, kind, p, q, r, n_r, n_i, ngrid, Ipi, U, A, Uf,
                                       Af, fhdr)
                       : ROMB_E_FORMAT;
    if (s != ROMB_OK) {
      for (int k2 = 0; k2 <= k; ++k2) free_model(c, c->roms[F.slot0 + k2]);
      fclose(f);
      return s;
    }
    RombRom& R = c->roms[F.slot0 + k];
    R.cluster = k;
    for (int d = 0, kk = k; d < 4; ++d, kk /= n_k) {
      R.lo4[d] = lohi[0] + h * (kk % n_k);
      R.hi4[d] = lohi[0] + h * (kk % n_k + 1);
    }
  }
  fclose(f);
  F.n_k = n_k;
  F.lo = lohi[0];
  F.hi = lohi[1];
  if (family_out) *family_out = family;
  return ROMB_OK;
}

// ---------------------------------------------------------------------------
// Lattice set-up: copies inputs, builds structural index tables
// ---------------------------------------------------------------------------
// The layout arrays of L on the host (empty when not given).
static romb_status read_layout(romb_ctx* c, const romb_lattice* L, std::vector<uint8_t>& pres,
                               std::vector<uint8_t>& clamp) {
  const size_t cells = (size_t)L->nx * L->ny;
  pres.clear();
  clamp.clear();
  const cudaMemcpyKind kind = L->mem == ROMB_MEM_HOST ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost;
  if (L->cell_present) {
    pres.resize(cells);
    ROMB_CUDA(cudaMemcpy(pres.data(), L->cell_present, cells, kind));
    for (uint8_t& v : pres) v = v ? 1 : 0;
  }
  if (L->edge_clamped) {
    clamp.resize(4 * cells);
    ROMB_CUDA(cudaMemcpy(clamp.data(), L->edge_clamped, 4 * cells, kind));
    for (uint8_t& v : clamp) v = v ? 1 : 0;
  }
  (void)c;
  return ROMB_OK;
}

static romb_status setup_lattice(romb_ctx* c, const romb_lattice* L, const std::vector<uint8_t>& pres,
                                 const std::vector<uint8_t>& clamp) {
  if (!L || L->nx < 1 || L->ny < 1 || L->p < 3 || L->p > ROMB_MAX_P || L->map_order < 1 ||
      L->map_order > 4 || (L->basis != 0 && L->basis != 1) || !L->ctrl || !L->mu || !L->family ||
      (L->mem != ROMB_MEM_HOST && L->mem != ROMB_MEM_DEVICE) || !(L->rho >= 0.0) || !(L->E > 0) ||
      !(L->nu > -1.0 && L->nu < 0.5))
    return ROMB_E_ARG;
  const long long cells = (long long)L->nx * L->ny;
  if (cells > (1LL << 22)) return ROMB_E_ARG;
  if (!pres.empty() && std::find(pres.begin(), pres.end(), (uint8_t)1) == pres.end()) {
    romb_set_error("lattice layout: no present cell");
    return ROMB_E_ARG;
  }
  const bool same = c->have_lattice && c->nx == L->nx && c->ny == L->ny && c->p == L->p &&
                    c->m == L->map_order && c->dmask == L->dirichlet_mask && c->h_present == pres &&
                    c->h_clamped == clamp;
  if (!same) {
    romb_free_lattice(c);
    return ROMB_E_STATE;
  }
  return ROMB_OK;
}

static romb_status build_tables(romb_ctx* c) {
  romb_status s;
  const int p = c->p, nx = c->nx, ny = c->ny, nB = c->nB, nU = c->nU, nI = c->nI;
  const long long cells = c->ncells;
  // local slot tables
  LocalTables T = make_local_tables(p);
  ROMB_CUDA(cudaMemcpy(c->d_islot, T.islot, sizeof(int) * nI, cudaMemcpyHostToDevice));
  ROMB_CUDA(cudaMemcpy(c->d_uslot, T.uslot, sizeof(int) * nU, cudaMemcpyHostToDevice));
  // skeleton map per cell, coarse map per cell
  std::vector<int> umap((size_t)cells * nU), cmap((size_t)cells * ROMB_NSLOT);
  const long long NH = (long long)(ny + 1) * (p * nx + 1);
  auto skel_id = [&](int gx, int gy) -> long long {   // grid node on a cell boundary -> skeleton node
    if (gy % p == 0) return (long long)(gy / p) * (p * nx + 1) + gx;
    return NH + ((long long)(gy / p) * (nx + 1) + gx / p) * (p - 1) + (gy % p - 1);
  };
  auto grid_xy = [&](long long cell, int* cx, int* cy) {
    const long long g = c->layout ? c->h_cell_grid[cell] : cell;
    *cx = (int)(g % nx);
    *cy = (int)(g / nx);
  };
  // layouts: the skeleton nodes that carry no unknown (clamped by the mask or
  // by a clamped cell edge, or on no present cell)
  std::vector<uint8_t> fixed;
  if (c->layout) {
    fixed.assign((size_t)c->nskel_nodes, 1);
    std::vector<uint8_t> clamped((size_t)c->nskel_nodes, 0);
    for (long long cell = 0; cell < cells; ++cell) {
      int cx, cy;
      grid_xy(cell, &cx, &cy);
      for (int u = 0; u < nU; u += 2) {
        const int k = T.uslot[u] / 2, a = k % (p + 1), b = k / (p + 1);
        fixed[skel_id(p * cx + a, p * cy + b)] = 0;
      }
      if (!c->h_clamped.empty())
        for (int e = 0; e < 4; ++e) {
          if (!c->h_clamped[4 * (size_t)(c->h_cell_grid[cell]) + e]) continue;
          for (int t = 0; t <= p; ++t) {
            const int a = e == 0 ? 0 : e == 1 ? p : t, b = e == 2 ? 0 : e == 3 ? p : t;
            clamped[skel_id(p * cx + a, p * cy + b)] = 1;
          }
        }
    }
    for (long long id = 0; id < c->nskel_nodes; ++id) {
      if (fixed[id]) continue;
      int gx, gy;
      if (id < NH) {
        gy = p * (int)(id / (p * nx + 1));
        gx = (int)(id % (p * nx + 1));
      } else {
        long long t = id - NH;
        const int b = (int)(t % (p - 1)) + 1;
        t /= (p - 1);
        gx = p * (int)(t % (nx + 1));
        gy = p * (int)(t / (nx + 1)) + b;
      }
      const bool side = ((c->dmask & 1) && gx == 0) || ((c->dmask & 2) && gx == p * nx) ||
                        ((c->dmask & 4) && gy == 0) || ((c->dmask & 8) && gy == p * ny);
      fixed[id] = side || clamped[id];
    }
    ROMB_CUDA(cudaMemcpy(c->d_node_fixed, fixed.data(), fixed.size(), cudaMemcpyHostToDevice));
  }
  auto dir_node = [&](int gx, int gy) {
    if (c->layout) return fixed[skel_id(gx, gy)] != 0;
    return ((c->dmask & 1) && gx == 0) || ((c->dmask & 2) && gx == p * nx) || ((c->dmask & 4) && gy == 0) ||
           ((c->dmask & 8) && gy == p * ny);
  };
  const long long NCV = 2LL * (nx + 1) * (ny + 1), NCH = 3LL * nx * (ny + 1);
  for (long long cell = 0; cell < cells; ++cell) {
    int cx, cy;
    grid_xy(cell, &cx, &cy);
    {
      for (int u = 0; u < nU; ++u) {
        const int k = T.uslot[u] / 2, comp = T.uslot[u] % 2;
        const int a = k % (p + 1), b = k / (p + 1);
        const int gx = p * cx + a, gy = p * cy + b;
        const long long id = skel_id(gx, gy);
        umap[cell * nU + u] = dir_node(gx, gy) ? -1 : (int)(2 * id + comp);
      }
      int* cm = &cmap[cell * ROMB_NSLOT];
      const int vxs[4] = {cx, cx + 1, cx, cx + 1}, vys[4] = {cy, cy, cy + 1, cy + 1};
      for (int v = 0; v < 4; ++v) {
        const bool d = dir_node(p * vxs[v], p * vys[v]);
        const long long base = 2LL * ((long long)vys[v] * (nx + 1) + vxs[v]);
        cm[2 * v] = d ? -1 : (int)base;
        cm[2 * v + 1] = d ? -1 : (int)(base + 1);
      }
      // edges: left (vx=cx), right (vx=cx+1), bottom (vy=cy), top (vy=cy+1);
      // an edge is clamped where its interior nodes are
      for (int e = 0; e < 4; ++e) {
        long long base;
        bool d;
        if (e < 2) {
          const int vx = cx + e;
          d = c->layout ? dir_node(p * vx, p * cy + 1)
                        : (vx == 0 && (c->dmask & 1)) || (vx == nx && (c->dmask & 2));
          base = NCV + NCH + 3LL * ((long long)cy * (nx + 1) + vx);
        } else {
          const int vy = cy + (e - 2);
          d = c->layout ? dir_node(p * cx + 1, p * vy)
                        : (vy == 0 && (c->dmask & 4)) || (vy == ny && (c->dmask & 8));
          base = NCV + 3LL * ((long long)vy * nx + cx);
        }
        for (int t = 0; t < 3; ++t) cm[8 + 3 * e + t] = d ? -1 : (int)(base + t);
      }
    }
  }
  (void)nB;
  ROMB_CUDA(cudaMemcpy(c->d_ucell_map, umap.data(), sizeof(int) * umap.size(), cudaMemcpyHostToDevice));
  ROMB_CUDA(cudaMemcpy(c->d_cmap, cmap.data(), sizeof(int) * cmap.size(), cudaMemcpyHostToDevice));
  c->ncoarse_all = NCV + NCH + 3LL * (nx + 1) * ny;
  {
    // owners of every coarse DoF, in increasing cell order
    std::vector<int> own((size_t)c->ncoarse_all * 4, -1);
    std::vector<int> cnt((size_t)c->ncoarse_all, 0);
    for (long long cell = 0; cell < cells; ++cell)
      for (int j = 0; j < ROMB_NSLOT; ++j) {
        const int g = cmap[cell * ROMB_NSLOT + j];
        if (g < 0) continue;
        if (cnt[g] >= 4) return ROMB_E_ARG;
        own[(size_t)g * 4 + cnt[g]++] = (int)(cell * ROMB_NSLOT + j);
      }
    ROMB_CUDA(cudaMemcpy(c->d_cowner, own.data(), sizeof(int) * own.size(), cudaMemcpyHostToDevice));
  }
  if ((s = coarse_build(c)) != ROMB_OK) return s;
  return ROMB_OK;
}

// Device buffers of one PCG lane for the current lattice (lane 0 with the
// lattice, further lanes on the first solve with several load sets).
static romb_status lane_buffers(romb_ctx* c, PcgLane& L) {
  if (L.have_bufs) return ROMB_OK;
  const long long cells = c->ncells;
  const long long nodes = (long long)(c->p * c->nx + 1) * (c->p * c->ny + 1);
  romb_status s;
#define A_(ptr, n)                                               \
  do {                                                           \
    if ((s = romb_alloc_t(c, &(ptr), (size_t)(n))) != ROMB_OK) return s; \
  } while (0)
  A_(L.d_f, c->nskel);
  A_(L.d_x, c->nskel);
  A_(L.d_r, c->nskel);
  A_(L.d_z, c->nskel);
  A_(L.d_pv, c->nskel);
  A_(L.d_q, c->nskel);
  A_(L.d_red, 4096);
  A_(L.d_fU, cells * c->nU);
  A_(L.d_fI, cells * c->nI);
  A_(L.d_cloc, cells * ROMB_NSLOT);
  A_(L.d_yloc, cells * c->nU);
  A_(L.d_u, 2 * nodes);
  A_(L.d_traction, 8 * 64);
  A_(L.d_coarse, 2 * c->ncoarse_all);
#undef A_
  if (&L != &c->lane[0] && (s = coarse_lane_buffers(c, &L.nd_ybuf, &L.nd_sbuf)) != ROMB_OK) return s;
  L.have_bufs = true;
  return ROMB_OK;
}

static romb_status alloc_lattice(romb_ctx* c, const romb_lattice* L, std::vector<uint8_t>& pres,
                                 std::vector<uint8_t>& clamp) {
  romb_status s;
  c->nx = L->nx;
  c->ny = L->ny;
  c->p = L->p;
  c->m = L->map_order;
  c->dmask = L->dirichlet_mask;
  c->ncells = L->nx * L->ny;
  c->layout = !pres.empty() || !clamp.empty();
  c->h_present.swap(pres);
  c->h_clamped.swap(clamp);
  std::vector<int> grid_cell;
  if (c->layout) {
    grid_cell.assign((size_t)c->ncells, -1);
    c->h_cell_grid.clear();
    for (int g = 0; g < c->ncells; ++g)
      if (c->h_present.empty() || c->h_present[g]) {
        grid_cell[g] = (int)c->h_cell_grid.size();
        c->h_cell_grid.push_back(g);
      }
    c->ncells = (int)c->h_cell_grid.size();
  }
  c->nB = (c->p + 1) * (c->p + 1);
  c->ndof = 2 * c->nB;
  c->nI = 2 * (c->p - 1) * (c->p - 1);
  c->nU = 8 * c->p;
  c->kpack = tri(c->ndof);
  c->upack = tri(c->nU);
  const long long cells = c->ncells;
  const int p = c->p, nx = c->nx, ny = c->ny;
  const long long nctrl = (long long)(c->m * nx + 1) * (c->m * ny + 1);
  c->nskel_nodes = (long long)(ny + 1) * (p * nx + 1) + (long long)ny * (nx + 1) * (p - 1);
  c->nskel = 2 * c->nskel_nodes;
  const long long nodes = (long long)(p * nx + 1) * (p * ny + 1);
#define A_(ptr, n)                                          \
  if ((s = romb_alloc_t(c, &(ptr), (size_t)(n))) != ROMB_OK) \
    return s;
  A_(c->d_ctrl, 2 * nctrl);
  A_(c->d_mu, 4 * cells);
  A_(c->d_family, cells);
  A_(c->d_flags, cells);
  A_(c->d_chat, cells * 9 * 16);
  A_(c->d_chat32, cells * 144);
  A_(c->d_theta, cells * 128);
  A_(c->d_theta_hi, cells * 128);
  A_(c->d_theta_lo, cells * 128);
  A_(c->d_famlist, cells);
  A_(c->d_slot, cells);
  A_(c->d_K, cells * c->kpack);
  A_(c->d_kdiag, cells * c->nU);
  A_(c->d_ktot, c->nskel);
  A_(c->d_LII, cells * tri(c->nI));
  A_(c->d_W, cells * (long long)c->nI * c->nU);
  A_(c->d_S, cells * (long long)c->nU * c->nU);
  A_(c->d_G, cells * (long long)c->nU * c->nU);
  A_(c->d_Phi, cells * (long long)c->nU * ROMB_NSLOT);
  A_(c->d_Psi, cells * (long long)c->nU * ROMB_NSLOT);
  A_(c->d_SCl, cells * ROMB_NSLOT * ROMB_NSLOT);
  A_(c->d_D, cells * c->nU);
  A_(c->d_efun, cells * 12LL * (c->p + 1));
  A_(c->d_eiv, cells * 4LL * (1 + 2 * ROMB_MAX_IV));
  A_(c->d_ucell_map, cells * c->nU);
  A_(c->d_islot, c->nI);
  A_(c->d_uslot, c->nU);
  A_(c->d_cmap, cells * ROMB_NSLOT);
  A_(c->d_red, 4096);
  A_(c->d_pcg_err, 1);
  if (c->layout) {
    const long long grid = (long long)nx * ny;
    A_(c->d_cell_grid, cells);
    A_(c->d_grid_cell, grid);
    A_(c->d_node_fixed, c->nskel_nodes);
    A_(c->d_stage, 4 * grid + (grid + 1) / 2);   // grid-indexed mu, then family
  }
#undef A_
  if (c->layout) {
    ROMB_CUDA(cudaMemcpy(c->d_cell_grid, c->h_cell_grid.data(), 4 * (size_t)cells, cudaMemcpyHostToDevice));
    ROMB_CUDA(cudaMemcpy(c->d_grid_cell, grid_cell.data(), 4 * grid_cell.size(), cudaMemcpyHostToDevice));
  }
  ROMB_CUDA(cudaMemsetAsync(c->d_pcg_err, 0, 4, c->stream));
  const long long ncoarse = 2LL * (nx + 1) * (ny + 1) + 3LL * nx * (ny + 1) + 3LL * (nx + 1) * ny;
  c->ncoarse_all = ncoarse;
  if ((s = lane_buffers(c, c->lane[0])) != ROMB_OK) return s;
  if ((s = romb_alloc_t(c, &c->d_cowner, 4 * ncoarse)) != ROMB_OK) return s;
  if ((s = build_tables(c)) != ROMB_OK) return s;
  c->have_lattice = true;
  return ROMB_OK;
}

// The present cells' thresholds and families out of the grid-indexed inputs.
__global__ void gather_present_kernel(long long n, const int* __restrict__ cell_grid, const double* __restrict__ mu_g,
                                      const int32_t* __restrict__ fam_g, double* __restrict__ mu,
                                      int32_t* __restrict__ fam) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long g = cell_grid[i];
    fam[i] = fam_g[g];
    for (int k = 0; k < 4; ++k) mu[4 * i + k] = mu_g[4 * g + k];
  }
}

// Copy (or reference) the lattice inputs and validate families.
static romb_status load_lattice(romb_ctx* c, const romb_lattice* L) {
  if (!L) return ROMB_E_ARG;
  std::vector<uint8_t> pres, clamp;
  romb_status s = read_layout(c, L, pres, clamp);
  if (s != ROMB_OK) return s;
  s = setup_lattice(c, L, pres, clamp);
  if (s == ROMB_E_ARG) return s;
  if (s == ROMB_E_STATE) {
    c->have_lattice = false;
    if ((s = alloc_lattice(c, L, pres, clamp)) != ROMB_OK) return s;
  }
  c->basis = L->basis;
  c->mem = L->mem;
  c->E = L->E;
  c->nu = L->nu;
  c->rho = L->rho;
  for (int i = 0; i < 8; ++i) c->traction[i] = L->traction ? (L->mem == ROMB_MEM_HOST ? L->traction[i] : 0.0) : 0.0;
  const long long cells = c->ncells;
  const long long nctrl = (long long)(c->m * c->nx + 1) * (c->m * c->ny + 1);
  const cudaMemcpyKind kind = L->mem == ROMB_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  cudaEventRecord(c->ev[12], c->stream);
  ROMB_CUDA(cudaMemcpyAsync(c->d_ctrl, L->ctrl, 16 * nctrl, kind, c->stream));
  if (!c->layout) {
    ROMB_CUDA(cudaMemcpyAsync(c->d_mu, L->mu, 32 * cells, kind, c->stream));
    ROMB_CUDA(cudaMemcpyAsync(c->d_family, L->family, 4 * cells, kind, c->stream));
  } else {
    // grid-indexed inputs through the staging buffer, then the present cells'
    const long long grid = (long long)c->nx * c->ny;
    int32_t* fam_g = reinterpret_cast<int32_t*>(c->d_stage + 4 * grid);
    ROMB_CUDA(cudaMemcpyAsync(c->d_stage, L->mu, 32 * grid, kind, c->stream));
    ROMB_CUDA(cudaMemcpyAsync(fam_g, L->family, 4 * grid, kind, c->stream));
    gather_present_kernel<<<c->sms, 256, 0, c->stream>>>(cells, c->d_cell_grid, c->d_stage, fam_g, c->d_mu,
                                                         c->d_family);
    ++c->launches;
    ROMB_CUDA(cudaGetLastError());
  }
  // the lattice's own traction is kept on the host (each solve copies its
  // load set to its lane)
  if (L->traction && L->mem == ROMB_MEM_DEVICE) {
    ROMB_CUDA(cudaMemcpyAsync(c->traction, L->traction, 64, cudaMemcpyDeviceToHost, c->stream));
    ROMB_CUDA(cudaStreamSynchronize(c->stream));
  }
  cudaEventRecord(c->ev[13], c->stream);
  ROMB_CUDA(cudaMemsetAsync(c->d_flags, 0, 4 * cells, c->stream));
  return ROMB_OK;
}

static float ms_between(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0.f;
  }
  return ms;
}

static romb_status check_flags(romb_ctx* c, int mask_bits) {
  // reduce the per-cell flags on the device; one int comes back
  int* d_any = (int*)c->d_red;
  ROMB_CUDA(cudaMemsetAsync(d_any, 0, sizeof(int), c->stream));
  romb_status s = launch_flag_or(c, d_any);
  if (s != ROMB_OK) return s;
  int h = 0;
  ROMB_CUDA(cudaMemcpyAsync(&h, d_any, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  ROMB_CUDA(cudaStreamSynchronize(c->stream));
  h &= mask_bits;
  if (h & ROMB_FLAG_OUT_OF_BOX) return ROMB_E_OUT_OF_BOX;
  if (h & ROMB_FLAG_BAD_MAP) return ROMB_E_BAD_MAP;
  if (h & ROMB_FLAG_NOT_SPD) return ROMB_E_NOT_SPD;
  if (h & ROMB_FLAG_NAN) return ROMB_E_NAN;
  return ROMB_OK;
}

extern "C" romb_status romb_assemble(romb_ctx* c, const romb_lattice* L, romb_precision prec) {
  if (!c || !L) return ROMB_E_ARG;
  if (prec != ROMB_FP64 && prec != ROMB_FP32_SPLIT && prec != ROMB_BF16_SPLIT) return ROMB_E_ARG;
  ROMB_CUDA(cudaSetDevice(c->device));
  bool any = false;
  for (auto& R : c->roms) any |= R.loaded;
  if (!any) return ROMB_E_STATE;
  romb_status s = load_lattice(c, L);
  if (s != ROMB_OK) return s;
  for (auto& R : c->roms)
    if (R.loaded && (R.p != c->p || R.kind != c->basis)) return ROMB_E_ARG;
  c->assembled = c->factored = c->solved = false;
  c->prec = prec;
  c->assembled_split = prec != ROMB_FP64;
  c->assembled_rom = true;
  cudaEventRecord(c->ev[0], c->stream);
  c->efun_ready = false;
  if ((s = launch_theta(c)) != ROMB_OK) return s;
  // the coarse DoFs' edge functionals depend on the geometry only
  if ((s = launch_edge_functionals(c)) != ROMB_OK) return s;
  cudaEventRecord(c->ev[1], c->stream);
  if (prec == ROMB_FP64) s = launch_assemble_fp64(c);
  else s = launch_assemble_tc(c);
  if (s != ROMB_OK) return s;
  cudaEventRecord(c->ev[2], c->stream);
  if ((s = check_flags(c, ROMB_FLAG_OUT_OF_BOX | ROMB_FLAG_BAD_MAP | ROMB_FLAG_NAN)) != ROMB_OK) return s;
  c->phase_ms[0] = ms_between(c->ev[0], c->ev[1]);
  c->phase_ms[1] = ms_between(c->ev[1], c->ev[2]);
  c->phase_ms[6] = ms_between(c->ev[12], c->ev[13]);
  c->assembled = true;
  return ROMB_OK;
}

extern "C" romb_status romb_assemble_host_K(romb_ctx* c, const romb_lattice* L, const double* K) {
  if (!c || !L || !K) return ROMB_E_ARG;
  ROMB_CUDA(cudaSetDevice(c->device));
  romb_status s = load_lattice(c, L);
  if (s != ROMB_OK) return s;
  c->assembled = c->factored = c->solved = false;
  c->assembled_split = false;
  c->assembled_rom = false;
  c->efun_ready = false;
  // pack the dense matrices on the device (upper triangle, row-major)
  double* dense = nullptr;
  const size_t nd = (size_t)c->ndof;
  if ((s = romb_alloc_t(c, &dense, (size_t)c->ncells * nd * nd)) != ROMB_OK) return s;
  ROMB_CUDA(cudaMemcpyAsync(dense, K, 8 * (size_t)c->ncells * nd * nd,
                            L->mem == ROMB_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                            c->stream));
  s = launch_pack_dense(c, dense);
  ROMB_CUDA(cudaStreamSynchronize(c->stream));
  romb_free_ptr(c, dense);
  if (s != ROMB_OK) return s;
  c->assembled = true;
  return ROMB_OK;
}

__global__ void to_f32_kernel(long long n, const double* __restrict__ src, float* __restrict__ dst) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

// Cells flagged not positive definite after a reduced-model assembly (at most
// fallback_max): their tensors I(mu) by the trainer's exact trimmed
// quadrature, K by the FP64 contraction against U' = [I_Pi; I(mu)] with theta
// = (rho, 1 - rho), flag NOT_SPD replaced by EXACT.  *applied: cells were redone.
static romb_status exact_fallback(romb_ctx* c, bool* applied) {
  *applied = false;
  if (c->fallback_max <= 0 || !c->assembled_rom) return ROMB_OK;
  const long long n = c->ncells;
  std::vector<int32_t> flags((size_t)n);
  ROMB_CUDA(cudaStreamSynchronize(c->stream));
  ROMB_CUDA(cudaMemcpy(flags.data(), c->d_flags, 4 * (size_t)n, cudaMemcpyDeviceToHost));
  std::vector<int> bad;
  for (long long i = 0; i < n; ++i)
    if ((flags[i] & ROMB_FLAG_NOT_SPD) && !(flags[i] & ROMB_FLAG_EXACT)) bad.push_back((int)i);
  if (bad.empty() || (int)bad.size() > c->fallback_max) return ROMB_OK;
  std::vector<double> mu(4 * (size_t)n);
  std::vector<int32_t> slot((size_t)n);
  ROMB_CUDA(cudaMemcpy(mu.data(), c->d_mu, 32 * (size_t)n, cudaMemcpyDeviceToHost));
  ROMB_CUDA(cudaMemcpy(slot.data(), c->d_slot, 4 * (size_t)n, cudaMemcpyDeviceToHost));
  romb_status s;
  double* dU = nullptr;
  int* dlist = nullptr;
  long long dU_n = 0;
  if ((s = romb_alloc_t(c, &dlist, 1)) != ROMB_OK) return s;
  for (int b : bad) {
    const RombRom& R = c->roms[slot[b]];
    romb_train_spec sp = {};
    sp.family = R.family;
    sp.basis = R.kind;
    sp.p = R.p;
    sp.q = R.q;
    sp.r = R.r;
    sp.n_r = R.n_r;
    sp.lo = R.lo4[0];
    sp.hi = R.hi4[0];
    const int nB = (R.p + 1) * (R.p + 1), nL = (R.q + 1) * (R.q + 1);
    const long long n_i = (long long)nB * nB * nL * 4;
    const std::vector<double> key = {(double)R.family, (double)R.kind, (double)R.p, (double)R.q, mu[4 * (size_t)b],
                                     mu[4 * (size_t)b + 1], mu[4 * (size_t)b + 2], mu[4 * (size_t)b + 3]};
    auto hit = c->exact_cache.find(key);
    if (hit == c->exact_cache.end()) {
      std::vector<double> I((size_t)n_i);
      if ((s = romb_train_snapshots_gpu(c->device, &sp, &mu[4 * (size_t)b], 1, I.data())) != ROMB_OK) return s;
      ROMB_CUDA(cudaSetDevice(c->device));
      // row 1 of U': I(mu) in the pair-major half layout (row 0: the model's I_Pi)
      std::vector<double> row((size_t)R.n_half);
      long long pr = 0;
      for (int k1 = 0; k1 < nB; ++k1)
        for (int k2 = k1; k2 < nB; ++k2, ++pr)
          for (int e = 0; e < nL * 4; ++e)
            row[(size_t)(pr * nL * 4 + e)] = I[(size_t)(((long long)k1 * nB + k2) * nL * 4 + e)];
      if (c->exact_cache.size() >= 256) c->exact_cache.clear();
      hit = c->exact_cache.emplace(key, std::move(row)).first;
    }
    const std::vector<double>& row = hit->second;
    if (dU_n < 2 * R.n_half) {
      if (dU) romb_free_ptr(c, dU);
      if ((s = romb_alloc_t(c, &dU, 2 * (size_t)R.n_half)) != ROMB_OK) return s;
      dU_n = 2 * R.n_half;
    }
    std::vector<double> th(128, 0.0);
    th[0] = c->rho;
    th[1] = 1.0 - c->rho;
    ROMB_CUDA(cudaMemcpy(dU, R.U64, 8 * (size_t)R.n_half, cudaMemcpyDeviceToDevice));
    ROMB_CUDA(cudaMemcpy(dU + R.n_half, row.data(), 8 * (size_t)R.n_half, cudaMemcpyHostToDevice));
    ROMB_CUDA(cudaMemcpy(c->d_theta + 128 * (size_t)b, th.data(), 8 * 128, cudaMemcpyHostToDevice));
    ROMB_CUDA(cudaMemcpy(dlist, &b, 4, cudaMemcpyHostToDevice));
    if ((s = launch_assemble_cells_fp64(c, dU, R.n_half, 2, dlist, 1)) != ROMB_OK) return s;
    ROMB_CUDA(cudaStreamSynchronize(c->stream));
  }
  if (dU) romb_free_ptr(c, dU);
  romb_free_ptr(c, dlist);
  for (long long i = 0; i < n; ++i) flags[i] &= ~ROMB_FLAG_NOT_SPD;
  for (int b : bad) flags[b] |= ROMB_FLAG_EXACT;
  ROMB_CUDA(cudaMemcpy(c->d_flags, flags.data(), 4 * (size_t)n, cudaMemcpyHostToDevice));
  *applied = true;
  return ROMB_OK;
}

extern "C" romb_status romb_set_exact_fallback(romb_ctx* c, int max_cells) {
  if (!c || max_cells < 0) return ROMB_E_ARG;
  c->fallback_max = max_cells;
  return ROMB_OK;
}

extern "C" romb_status romb_factor(romb_ctx* c) {
  if (!c) return ROMB_E_ARG;
  if (!c->assembled) return ROMB_E_STATE;
  ROMB_CUDA(cudaSetDevice(c->device));
  romb_status s;
  for (PcgLane& L : c->lane)   // the captured PCG loops hold this factorisation's launch shapes
    if (L.graph) {
      cudaGraphExecDestroy(L.graph);
      L.graph = nullptr;
    }
  // the split-precision forms apply the preconditioner in FP32 (the operator
  // S and the PCG vectors stay FP64): D F D, Phi and the coarse solve's B
  c->pre32 = c->precond_mode < 0 ? c->assembled_split : c->precond_mode == 1;
  for (int attempt = 0;; ++attempt) {
    cudaEventRecord(c->ev[3], c->stream);
    if ((s = launch_ktot(c)) != ROMB_OK) return s;
    if ((s = launch_factor(c)) != ROMB_OK) return s;
    cudaEventRecord(c->ev[4], c->stream);
    s = coarse_factor(c);
    if (s == ROMB_OK && c->pre32) {
      const long long nG = (long long)c->ncells * c->nU * c->nU, nP = (long long)c->ncells * c->nU * ROMB_NSLOT;
      if (!c->d_G32 && (s = romb_alloc_t(c, &c->d_G32, (size_t)nG)) != ROMB_OK) return s;
      if (!c->d_Phi32 && (s = romb_alloc_t(c, &c->d_Phi32, (size_t)nP)) != ROMB_OK) return s;
      to_f32_kernel<<<4 * c->sms, 256, 0, c->stream>>>(nG, c->d_G, c->d_G32);
      to_f32_kernel<<<4 * c->sms, 256, 0, c->stream>>>(nP, c->d_Phi, c->d_Phi32);
      c->launches += 2;
      ROMB_CUDA(cudaGetLastError());
    }
    cudaEventRecord(c->ev[5], c->stream);
    if (s == ROMB_OK) s = check_flags(c, ROMB_FLAG_NOT_SPD | ROMB_FLAG_NAN);
    if (s == ROMB_E_NOT_SPD && attempt == 0) {   // cells whose reduced K lost definiteness
      bool applied = false;
      romb_status s2 = exact_fallback(c, &applied);
      if (s2 != ROMB_OK) return s2;
      if (applied) continue;
    }
    if (s != ROMB_OK) return s;
    break;
  }
  c->phase_ms[2] = ms_between(c->ev[3], c->ev[4]);
  c->phase_ms[3] = ms_between(c->ev[4], c->ev[5]);
  c->factored = true;
  return ROMB_OK;
}

extern "C" romb_status romb_bddc_solve(romb_ctx* c, int nrhs, const double* traction_sets, double rtol,
                                       int maxit, double* u_out, int* iters_out, double* relres_out) {
  if (!c || !u_out || nrhs < 1 || !(rtol > 0) || maxit < 1) return ROMB_E_ARG;
  if (!traction_sets && nrhs != 1) return ROMB_E_ARG;
  if (!c->factored) return ROMB_E_STATE;
  if (c->body[0] != 0.0 || c->body[1] != 0.0) {   // body forces need the volume part of the force models
    if (c->load_form != ROMB_LOADS_REDUCED) {
      romb_set_error("body forces: select ROMB_LOADS_REDUCED (romb_set_load_form)");
      return ROMB_E_STATE;
    }
    for (int f = 0; f < ROMB_MAX_MODELS; ++f)
      if (c->famcount[f] > 0 && c->roms[f].force_nf != 4 * (c->p + 1) * (c->q + 1) + c->nB * c->nL) {
        romb_set_error("body forces: a reduced model in use has no volume part in its force model");
        return ROMB_E_STATE;
      }
  }
  if (c->load_form == ROMB_LOADS_REDUCED) {   // checked before any work is enqueued
    if (!c->assembled_rom) {
      romb_set_error("reduced loads: the cell matrices were not assembled from the reduced models");
      return ROMB_E_STATE;
    }
    for (int f = 0; f < ROMB_MAX_MODELS; ++f)
      if (c->famcount[f] > 0 &&
          (!c->roms[f].force_U || c->roms[f].force_rf > 128 ||
           (c->roms[f].force_nf != 4 * (c->p + 1) * (c->q + 1) &&
            c->roms[f].force_nf != 4 * (c->p + 1) * (c->q + 1) + c->nB * c->nL))) {
        romb_set_error("reduced loads: the reduced model of a family in use has no force model of this degree");
        return ROMB_E_STATE;
      }
  }
  ROMB_CUDA(cudaSetDevice(c->device));
  const long long nodes = (long long)(c->p * c->nx + 1) * (c->p * c->ny + 1);
  const bool dev = c->mem == ROMB_MEM_DEVICE;
  romb_status s;
  // Load sets run concurrently on up to ROMB_MAX_LANES lanes (each its own
  // streams, vectors and captured PCG loop, all reading the one factorisation),
  // in waves; set k goes to lane k % nl, and the waves run from the last to
  // the first, so that lane 0 ends on set 0, whose state the compliance
  // gradient reads.  Two host synchronisations per wave: after ||f|| and at
  // the end.
  const int nl = std::min(nrhs, ROMB_MAX_LANES);
  for (int k = 1; k < nl; ++k) {
    if ((s = pcg_lane_streams(c, c->lane[k], false)) != ROMB_OK) return s;
    if ((s = lane_buffers(c, c->lane[k])) != ROMB_OK) return s;
  }
  romb_status worst = ROMB_OK;
  double rec_ms = 0.0;
  c->phase_ms[6] = 0.0;
  cudaEventRecord(c->ev[6], c->stream);
  const int nwaves = (nrhs + nl - 1) / nl;
  for (int w = nwaves - 1; w >= 0; --w) {
    const int k0 = w * nl, kn = std::min(nrhs, k0 + nl) - k0;
    for (int j = 0; j < kn; ++j) {
      PcgLane& L = c->lane[j];
      if (j > 0) {   // lanes start after everything before this call on the context stream
        ROMB_CUDA(cudaEventRecord(c->ev[14], c->stream));
        ROMB_CUDA(cudaStreamWaitEvent(L.stream, c->ev[14], 0));
      }
      const double* tr = traction_sets ? traction_sets + 8 * (k0 + j) : c->traction;
      if ((s = pcg_begin(c, L, tr, traction_sets && dev)) != ROMB_OK) return s;
    }
    for (int j = 0; j < kn; ++j) ROMB_CUDA(cudaStreamSynchronize(c->lane[j].stream));
    for (int j = 0; j < kn; ++j) {
      PcgLane& L = c->lane[j];
      L.nf = sqrt(L.h_red[1]);
      if ((s = pcg_finish(c, L, rtol, maxit)) != ROMB_OK) return s;
      double* dst = u_out + 2 * nodes * (k0 + j);
      ROMB_CUDA(cudaMemcpyAsync(dst, L.d_u, 16 * nodes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                L.stream));
    }
    for (int j = 0; j < kn; ++j) {
      PcgLane& L = c->lane[j];
      ROMB_CUDA(cudaStreamSynchronize(L.stream));
      int it = 0;
      double rel = 0.0;
      s = pcg_result(c, L, rtol, maxit, &it, &rel);
      if (s != ROMB_OK && s != ROMB_E_NOT_CONVERGED) return s;
      if (s == ROMB_E_NOT_CONVERGED) worst = s;
      if (iters_out) iters_out[k0 + j] = it;
      if (relres_out) relres_out[k0 + j] = rel;
      rec_ms += ms_between(L.ev0, L.ev1);
    }
  }
  // the lanes' work is complete (synchronised above); the end event on the
  // context stream closes the wall time of the whole call
  cudaEventRecord(c->ev[7], c->stream);
  ROMB_CUDA(cudaStreamSynchronize(c->stream));
  // [4]: wall time of the solves (loads, PCG, recovery, output copies) of all
  // load sets; [5]: the recoveries' own time (summed over sets when nrhs = 1
  // this is one recovery)
  c->phase_ms[5] = rec_ms;
  c->phase_ms[4] = ms_between(c->ev[6], c->ev[7]) - (nrhs == 1 ? rec_ms : 0.0);
  c->phase_ms[7] = c->phase_ms[0] + c->phase_ms[1] + c->phase_ms[2] + c->phase_ms[3] + c->phase_ms[4] +
                   (nrhs == 1 ? c->phase_ms[5] : 0.0);
  c->solved = true;
  return worst;
}

__global__ void sum4_kernel(const double* __restrict__ dmu, long long n, double* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = dmu[4 * i] + dmu[4 * i + 1] + dmu[4 * i + 2] + dmu[4 * i + 3];
}

extern "C" romb_status romb_compliance_grad(romb_ctx* c, double* compliance, double* dc_dctrl, double* dc_dR,
                                            double* dc_dmu) {
  if (!c || !compliance || !dc_dctrl) return ROMB_E_ARG;
  if (!c->solved || !c->assembled_rom) return ROMB_E_STATE;
  if (c->lane[0].body_on || c->load_form != ROMB_LOADS_QUADRATURE) {
    romb_set_error("compliance gradient: only for the quadrature traction loads without body forces");
    return ROMB_E_STATE;
  }
  if (c->layout) {
    romb_set_error("compliance gradient: only for the full rectangle of cells");
    return ROMB_E_STATE;
  }
  ROMB_CUDA(cudaSetDevice(c->device));
  romb_status s;
  const long long nctrl = (long long)(c->m * c->nx + 1) * (c->m * c->ny + 1);
  if (!c->d_gdmu) {
    if ((s = romb_alloc_t(c, &c->d_gdmu, 4 * (size_t)c->ncells)) != ROMB_OK) return s;
    if ((s = romb_alloc_t(c, &c->d_gdctrl, 2 * (size_t)nctrl)) != ROMB_OK) return s;
  }
  // c = f^T u on the skeleton (no interior forces)
  if ((s = romb_dot(c, c->lane[0].d_f, c->lane[0].d_x, c->nskel, c->d_red + 8)) != ROMB_OK) return s;
  ROMB_CUDA(cudaMemcpyAsync(c->h_red + 2, c->d_red + 8, 8, cudaMemcpyDeviceToHost, c->stream));
  const bool dev = c->mem == ROMB_MEM_DEVICE;
  double* d_ctrl_out = dev ? dc_dctrl : c->d_gdctrl;
  double* d_mu_out = (dev && dc_dmu) ? dc_dmu : c->d_gdmu;
  if ((s = launch_grad(c, d_ctrl_out, d_mu_out)) != ROMB_OK) return s;
  if (dc_dR) {
    double* d_r_out = dev ? dc_dR : c->d_gdctrl + 0;   // host case handled below
    if (dev) {
      sum4_kernel<<<c->sms, 256, 0, c->stream>>>(d_mu_out, c->ncells, d_r_out); ++c->launches;
      ROMB_CUDA(cudaGetLastError());
    }
  }
  if (!dev) {
    ROMB_CUDA(cudaMemcpyAsync(dc_dctrl, c->d_gdctrl, 16 * nctrl, cudaMemcpyDeviceToHost, c->stream));
    std::vector<double> dmu(4 * (size_t)c->ncells);
    ROMB_CUDA(cudaMemcpyAsync(dmu.data(), c->d_gdmu, 32 * (size_t)c->ncells, cudaMemcpyDeviceToHost, c->stream));
    ROMB_CUDA(cudaStreamSynchronize(c->stream));
    if (dc_dmu) memcpy(dc_dmu, dmu.data(), 32 * (size_t)c->ncells);
    if (dc_dR)
      for (long long i = 0; i < c->ncells; ++i) dc_dR[i] = dmu[4 * i] + dmu[4 * i + 1] + dmu[4 * i + 2] + dmu[4 * i + 3];
  }
  ROMB_CUDA(cudaStreamSynchronize(c->stream));
  *compliance = c->h_red[2];
  return ROMB_OK;
}

extern "C" romb_status romb_set_body_force(romb_ctx* c, double bx, double by) {
  if (!c || !std::isfinite(bx) || !std::isfinite(by)) return ROMB_E_ARG;
  c->body[0] = bx;
  c->body[1] = by;
  return ROMB_OK;
}

extern "C" romb_status romb_set_load_form(romb_ctx* c, int form) {
  if (!c || (form != ROMB_LOADS_QUADRATURE && form != ROMB_LOADS_REDUCED)) return ROMB_E_ARG;
  c->load_form = form;
  return ROMB_OK;
}

extern "C" romb_status romb_set_precond_precision(romb_ctx* c, int mode) {
  if (!c || mode < ROMB_PRECOND_AUTO || mode > ROMB_PRECOND_FP32) return ROMB_E_ARG;
  c->precond_mode = mode;
  return ROMB_OK;
}

extern "C" romb_status romb_stats(romb_ctx* c, double* phase_ms, int* flags_out) {
  if (!c) return ROMB_E_ARG;
  if (phase_ms) memcpy(phase_ms, c->phase_ms, sizeof(c->phase_ms));
  if (flags_out) {
    if (!c->have_lattice) return ROMB_E_STATE;
    ROMB_CUDA(cudaSetDevice(c->device));
    ROMB_CUDA(cudaMemcpyAsync(flags_out, c->d_flags, 4 * (size_t)c->ncells, cudaMemcpyDeviceToHost, c->stream));
    ROMB_CUDA(cudaStreamSynchronize(c->stream));
  }
  return ROMB_OK;
}

extern "C" long long romb_launch_count(romb_ctx* c) { return c ? c->launches : -1; }

extern "C" size_t romb_field_bytes(romb_ctx* c, int field) {
  if (!c || !c->have_lattice) return 0;
  const size_t cells = (size_t)c->ncells, nU = (size_t)c->nU;
  int kmax = 0;
  for (auto& R : c->roms)
    if (R.loaded) kmax = std::max(kmax, R.n_r + 1);
  switch (field) {
    case ROMB_FIELD_CHAT: return cells * 9 * 16 * 8;
    case ROMB_FIELD_THETA: return cells * (size_t)kmax * 8;
    case ROMB_FIELD_K: return cells * (size_t)c->kpack * 8;
    case ROMB_FIELD_S: return cells * tri(nU) * 8;
    case ROMB_FIELD_PSI: return cells * nU * ROMB_NSLOT * 8;
    case ROMB_FIELD_SC_LOCAL: return cells * ROMB_NSLOT * ROMB_NSLOT * 8;
    case ROMB_FIELD_D: return cells * nU * 8;
    case ROMB_FIELD_FINE: return cells * tri(nU) * 8;
    case ROMB_FIELD_FLAGS: return cells * 4;
    case ROMB_FIELD_LOADS: return c->lane[0].d_fU ? cells * nU * 8 : 0;
  }
  return 0;
}

extern "C" romb_status romb_read(romb_ctx* c, int field, void* out, size_t bytes) {
  if (!c || !out) return ROMB_E_ARG;
  const size_t need = romb_field_bytes(c, field);
  if (need == 0 || bytes != need) return ROMB_E_ARG;
  ROMB_CUDA(cudaSetDevice(c->device));
  ROMB_CUDA(cudaStreamSynchronize(c->stream));
  const size_t cells = (size_t)c->ncells, nU = (size_t)c->nU;
  switch (field) {
    case ROMB_FIELD_CHAT: ROMB_CUDA(cudaMemcpy(out, c->d_chat, bytes, cudaMemcpyDeviceToHost)); break;
    case ROMB_FIELD_THETA: {
      const size_t k = bytes / (cells * 8);
      std::vector<double> tmp(cells * 128);
      ROMB_CUDA(cudaMemcpy(tmp.data(), c->d_theta, tmp.size() * 8, cudaMemcpyDeviceToHost));
      for (size_t i = 0; i < cells; ++i) memcpy((double*)out + i * k, &tmp[i * 128], 8 * k);
      break;
    }
    case ROMB_FIELD_K: ROMB_CUDA(cudaMemcpy(out, c->d_K, bytes, cudaMemcpyDeviceToHost)); break;
    case ROMB_FIELD_S:
    case ROMB_FIELD_FINE: {
      std::vector<double> full(cells * nU * nU);
      ROMB_CUDA(cudaMemcpy(full.data(), field == ROMB_FIELD_S ? c->d_S : c->d_G, full.size() * 8,
                           cudaMemcpyDeviceToHost));
      double* o = (double*)out;
      for (size_t i = 0; i < cells; ++i)
        for (size_t r = 0, t = 0; r < nU; ++r)
          for (size_t q = r; q < nU; ++q, ++t) o[i * tri(nU) + t] = full[i * nU * nU + r * nU + q];
      break;
    }
    case ROMB_FIELD_PSI: ROMB_CUDA(cudaMemcpy(out, c->d_Psi, bytes, cudaMemcpyDeviceToHost)); break;
    case ROMB_FIELD_SC_LOCAL: ROMB_CUDA(cudaMemcpy(out, c->d_SCl, bytes, cudaMemcpyDeviceToHost)); break;
    case ROMB_FIELD_D: ROMB_CUDA(cudaMemcpy(out, c->d_D, bytes, cudaMemcpyDeviceToHost)); break;
    case ROMB_FIELD_FLAGS: ROMB_CUDA(cudaMemcpy(out, c->d_flags, bytes, cudaMemcpyDeviceToHost)); break;
    case ROMB_FIELD_LOADS: ROMB_CUDA(cudaMemcpy(out, c->lane[0].d_fU, bytes, cudaMemcpyDeviceToHost)); break;
    default: return ROMB_E_ARG;
  }
  return ROMB_OK;
}
