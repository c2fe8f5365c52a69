// C ABI of the BSE hot path: context set-up, screened-integral build, Liouville
// operator application and block Davidson (declared in include/bse.h).
#include "bse.h"
#include "kernels.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <queue>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

using namespace bse;

// ---------------------------------------------------------------------------------
// region profiler: CUDA events on the context stream around instrumented regions
// ---------------------------------------------------------------------------------
struct Prof {
  bool on = false;
  struct Pending { int id; cudaEvent_t a, b; double bytes, flops; };
  std::vector<Pending> pend;
  std::vector<bse_prof_entry> acc;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get() {
    if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  int id_of(const char* name) {
    for (size_t i = 0; i < acc.size(); ++i)
      if (!strncmp(acc[i].name, name, sizeof(acc[i].name))) return (int)i;
    bse_prof_entry e{};
    strncpy(e.name, name, sizeof(e.name) - 1);
    acc.push_back(e);
    return (int)acc.size() - 1;
  }
  void resolve() {   // call after the stream has been synchronised
    for (auto& p : pend) {
      float ms = 0;
      if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) acc[p.id].ms += ms;
      acc[p.id].calls += 1;
      acc[p.id].bytes += p.bytes;
      acc[p.id].flops += p.flops;
      pool.push_back(p.a); pool.push_back(p.b);
    }
    pend.clear();
  }
  ~Prof() {
    for (auto& p : pend) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

// opaque storage for a TMA tensor map (CUtensorMap is 128 bytes, 64-byte aligned)
struct TMap { alignas(64) unsigned char b[128]; };
// bf16 hi/lo split of an operand with its two tensor maps
struct Split {
  void* hi = nullptr;
  void* lo = nullptr;
  long rows = 0, cols = 0, ld = 0;
  TMap mhi, mlo;
};

struct bse_ctx {
  Prof prof;
  // tensor-core (BF16x3) operands of the mixed path
  bool tc_ok = false;
  Split psi_s, psiT_s, pdep_s, pdepT_s, qpsi_s, qpsiT_s;
  // explicit QP terms of D (Eq. ham): conduction KS states n_occ+1..N_QP and their delta_c
  int n_qc = 0;
  double *qpsi64 = nullptr, *qdelta = nullptr;
  float* qpsi32 = nullptr;
  // occupied energies as a matrix after a localising rotation (bse_localize): E = U^T diag(eps) U;
  // its diagonal sits in eps / esh, the rest (E_off) enters D as - sum_w E_vw a_w
  bool has_emat = false;
  double* eoff64 = nullptr;
  float* eoff32 = nullptr;
  double spread0 = 0, spread1 = 0;
  void *ws_ahi = nullptr, *ws_alo = nullptr, *ws_bhi = nullptr, *ws_blo = nullptr;
  long ws_split_rows = 0;
  // TMA maps of the split workspace, by (base pointer, leading dimension); they span the
  // workspace's full row capacity, so they stay valid until it is reallocated
  std::map<std::pair<const void*, long>, TMap> ws_maps;
  int* d_err = nullptr;
  // polls of each tensor-core pipeline wait before it gives up (BSE_TC_WAIT_LIMIT; -1 default)
  long long tc_wait_limit = -1;
  // learned preconditioner: inference weights and training samples
  float* lp_params = nullptr;
  int* d_bad = nullptr;
  long lp_ns = 0;                      // samples held
  int lp_cg_iters = 0;                 // CG iterations of the last exact-target solve
  double *lp_r = nullptr, *lp_t = nullptr, *lp_theta = nullptr, *lp_rn2 = nullptr, *lp_tn2 = nullptr;
  double* lp_u = nullptr;              // Ritz vectors of the collected samples (null for caller samples)
  // problem
  int N = 0;
  long n3 = 0;
  double L = 0, omega = 0, scissor = 0, thr_in = 0, v0 = 0;
  int n_half = 0, n_pw = 0, n_occ = 0, n_pdep = 0, spin = 0, prec = 0;
  int64_t keep_pairs = 0;
  cudaStream_t st = nullptr;
  // caller-supplied device allocator (both null: cudaMallocAsync on the context stream)
  bse_alloc_fn ua = nullptr;
  bse_free_fn uf = nullptr;
  void* uu = nullptr;
  std::string err = "no error";
  std::vector<double> g2p_h, eps_h, O_h;
  std::vector<double> gcart_h;  // [3][n_pw]: Cartesian G components per packed coordinate
  // per spin channel and packed coordinate j: sum_{v in channel} psi_v(j)^2 (occupied weight)
  std::vector<double> occw_h;
  int n_up = 0;                // spin-polarised: orbitals [0, n_up) up, [n_up, n_occ) down; 0 closed shell
  int chan(int v) const { return (n_up > 0 && v >= n_up) ? 1 : 0; }
  // K1e factor of Eq. (k1e): 2 closed-shell singlet, 0 triplet, 1 per spin-orbital when polarised
  double k1e_factor() const { return n_up > 0 ? 1.0 : (spin == 0 ? 2.0 : 0.0); }
  std::vector<int32_t> pv_h, pw_h;
  double thr = 0;
  bool tau_ready = false;
  // device, common
  int *gpos = nullptr, *gneg = nullptr;
  SphereMap sph;             // column-ordered sphere for the pruned transforms
  double *g2p = nullptr, *eps = nullptr, *f = nullptr;
  // 1/2|G|^2 per packed coordinate and Delta - eps_v per orbital, in both precisions
  double *g2h64 = nullptr, *esh64 = nullptr;
  float *g2h32 = nullptr, *esh32 = nullptr;
  double2* tw64 = nullptr;
  float2* tw32 = nullptr;
  // FP64 masters and FP32 copies
  double *psi64 = nullptr, *pdep64 = nullptr, *vloc64 = nullptr, *upsi64 = nullptr;
  float *psi32 = nullptr, *pdep32 = nullptr, *vloc32 = nullptr, *upsi32 = nullptr;
  // pairs / tau
  int *nbr_ptr = nullptr, *nbr_w = nullptr, *nbr_p = nullptr, *pv = nullptr, *pw = nullptr;
  // row blocks of four orbitals: union of the rows' neighbours (one entry each)
  int *bptr = nullptr, *bw = nullptr;
  int2* tslot = nullptr;     // per pair: the entry slots (4 e + row) that hold its tau
  int n_rblocks = 0;
  int64_t n_ent = 0;
  bool tau_entry = false;    // tau stored entry-major for the tiled K1d kernel
  // tau stored once per pair for the symmetric-layout tiled kernel (when the entry-major one
  // would not fit): upper entries and transposed tiles of every row block
  bool tau_sym = false;
  int tau_layout = -1;       // layout taken by the first build (0 per pair, 1 entry-major, 2 once per pair)
  int *ubptr = nullptr, *ubw = nullptr, *utptr = nullptr, *utinfo = nullptr;
  int4* utent = nullptr;
  int2* uslot = nullptr;
  int64_t n_ent_u = 0;
  std::map<int, int> k1d_var_sym;
  // K1d tile variant per block width n_vec, chosen by the autotuner (absent: not tuned yet)
  std::map<int, int> k1d_var;
  int k1d_force = 0;         // BSE_K1D_VARIANT: one variant for every width, no tuning
  int k1d_force_sym = 0;     // BSE_K1D_SYM_VARIANT: the same for tau stored once per pair
  bool autotune = true;
  int64_t n_pairs = 0, nnz = 0;
  void* tau = nullptr;       // entry-major (tau_entry) or per pair, point-tiled
  // operator workspace
  void *ws_a = nullptr, *ws_r = nullptr, *ws_h = nullptr, *ws_c = nullptr;
  long ws_vecs = 0;
  size_t ws_budget = 0;
  std::vector<void*> allocs;
};

namespace {

int fail(bse_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}
int cuda_fail(bse_ctx* c, cudaError_t e, const char* what) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
  if (c) c->err = buf;
  return (e == cudaErrorMemoryAllocation) ? BSE_ERR_OOM : BSE_ERR_CUDA;
}
#define CK(call)                                             \
  do {                                                       \
    cudaError_t _e = (call);                                 \
    if (_e != cudaSuccess) return cuda_fail(c, _e, #call);   \
  } while (0)

// Every device buffer of a context comes from here: from the caller's allocator when one
// was given to bse_create, else stream-ordered on the context stream, so independent
// contexts (e.g. a batch of systems on separate streams) never wait on each other's
// allocations.
template <typename T>
int dalloc(bse_ctx* c, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  const size_t bytes = count * sizeof(T);
  if (c->ua) {
    void* q = c->ua(bytes, c->uu);
    if (!q || ((uintptr_t)q & 255)) {
      if (q) c->uf(q, c->uu);
      char buf[256];
      snprintf(buf, sizeof(buf), "the caller's allocator %s for %zu bytes",
               q ? "returned a block not aligned to 256 bytes" : "returned NULL", bytes);
      c->err = buf;
      return BSE_ERR_OOM;
    }
    *p = (T*)q;
  } else {
    cudaError_t e = cudaMallocAsync((void**)p, bytes, c->st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *p = nullptr;
      char buf[256];
      snprintf(buf, sizeof(buf), "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
      c->err = buf;
      return BSE_ERR_OOM;
    }
  }
  c->allocs.push_back(*p);
  return BSE_OK;
}
void dfree_raw(bse_ctx* c, void* p) {
  if (c->uf) c->uf(p, c->uu);
  else cudaFreeAsync(p, c->st);
}
void dfree(bse_ctx* c, void* p) {
  if (!p) return;
  auto it = std::find(c->allocs.begin(), c->allocs.end(), p);
  if (it != c->allocs.end()) c->allocs.erase(it);
  dfree_raw(c, p);
}
struct Scope {
  bse_ctx* c; int id = -1; cudaEvent_t a = nullptr; double bytes, flops;
  Scope(bse_ctx* c_, const char* name, double b, double f) : c(c_), bytes(b), flops(f) {
    if (!c->prof.on) return;
    id = c->prof.id_of(name);
    a = c->prof.get();
    cudaEventRecord(a, c->st);
  }
  ~Scope() {
    if (id < 0) return;
    cudaEvent_t b = c->prof.get();
    cudaEventRecord(b, c->st);
    c->prof.pend.push_back({id, a, b, bytes, flops});
  }
};
inline double fft_flops(long n3, long grids) { return 5.0 * (double)n3 * std::log2((double)n3) * (double)grids; }

#define CA(expr)                    \
  do {                              \
    int _r = (expr);                \
    if (_r != BSE_OK) return _r;    \
  } while (0)

bool all_finite(const double* x, long n) { return finite_check_host(x, n); }

inline long pad8(long x) { return (x + 7) / 8 * 8; }

// split a resident FP64 matrix [rows x cols] (optionally transposed) into bf16 hi/lo with maps
int make_split64(bse_ctx* c, Split& sp, const double* X, long rows, long cols, bool transpose) {
  sp.rows = transpose ? cols : rows;
  sp.cols = transpose ? rows : cols;
  sp.ld = pad8(sp.cols);
  unsigned short *h, *l;
  CA(dalloc(c, &h, (size_t)sp.rows * sp.ld));
  CA(dalloc(c, &l, (size_t)sp.rows * sp.ld));
  sp.hi = h; sp.lo = l;
  CK(bf16_split64(X, rows, (int)cols, cols, h, l, sp.ld, transpose, c->st));
  // maps span the zero-padded width so the inner extent is at least 16 bytes
  if (!tc_make_map(sp.mhi.b, sp.hi, sp.rows, sp.ld, sp.ld) || !tc_make_map(sp.mlo.b, sp.lo, sp.rows, sp.ld, sp.ld))
    return fail(c, BSE_ERR_CUDA, "TMA tensor map creation failed");
  return BSE_OK;
}

// workspace for the per-call splits: A operand (K = n_pw) and the small-K operand
int ensure_split_ws(bse_ctx* c, long rows) {
  if (rows <= c->ws_split_rows) return BSE_OK;
  c->ws_maps.clear();
  dfree(c, c->ws_ahi); dfree(c, c->ws_alo); dfree(c, c->ws_bhi); dfree(c, c->ws_blo);
  c->ws_ahi = c->ws_alo = c->ws_bhi = c->ws_blo = nullptr;
  c->ws_split_rows = 0;
  const long ldk = pad8(c->n_pw), lds = pad8(std::max(std::max(c->n_occ, c->n_qc), std::max(1, c->n_pdep)));
  unsigned short* p;
  CA(dalloc(c, &p, (size_t)rows * ldk)); c->ws_ahi = p;
  CA(dalloc(c, &p, (size_t)rows * ldk)); c->ws_alo = p;
  CA(dalloc(c, &p, (size_t)rows * lds)); c->ws_bhi = p;
  CA(dalloc(c, &p, (size_t)rows * lds)); c->ws_blo = p;
  c->ws_split_rows = rows;
  return BSE_OK;
}

// out[M x N] = alpha * X[M x K] * B^T + beta * out  with B given by a resident split (N x K)
int tc_product(bse_ctx* c, const float* X, long M, long K, long ldx, const Split& B, bool small_k_slot,
               float* out, long ldo, double alpha, double beta) {
  CA(ensure_split_ws(c, M));
  const long ld = pad8(K);
  void* hi = small_k_slot ? c->ws_bhi : c->ws_ahi;
  void* lo = small_k_slot ? c->ws_blo : c->ws_alo;
  CK(bf16_split(X, M, (int)K, ldx, hi, lo, ld, c->st));
  // maps over the workspace's full capacity, built once: rows M.. of the last tile read
  // stale split data, whose output rows are never written
  auto ws_map = [&](const void* p) -> const TMap* {
    const auto key = std::make_pair(p, ld);
    auto it = c->ws_maps.find(key);
    if (it != c->ws_maps.end()) return &it->second;
    TMap m;
    if (!tc_make_map(m.b, p, c->ws_split_rows, ld, ld)) return nullptr;
    return &(c->ws_maps[key] = m);
  };
  const TMap* mhp = ws_map(hi);
  const TMap* mlp = ws_map(lo);
  if (!mhp || !mlp) return fail(c, BSE_ERR_CUDA, "TMA tensor map creation failed");
  const TMap& mh = *mhp;
  const TMap& ml = *mlp;
  const long tiles = ((M + 127) / 128) * ((B.rows + 127) / 128);
  const long kt = (K + 63) / 64;
  int splits = 1;
  if (beta == 0.0 && tiles < 2 * 152) splits = (int)std::min<long>(std::max<long>(1, 304 / tiles), std::max<long>(1, kt / 4));
  CK(tc_gemm_bf16x3(mh.b, ml.b, B.mhi.b, B.mlo.b, (int)M, (int)B.rows, (int)K, alpha, beta, out, ldo,
                    splits, c->d_err, c->st, c->tc_wait_limit));
  return BSE_OK;
}

// threshold rule of the pair list (same reading as documented in bse.h)
double choose_threshold(const std::vector<double>& O, int n, double thr, int64_t keep) {
  if (thr > 0) return thr;
  std::vector<double> off;
  off.reserve((size_t)n * (n - 1) / 2);
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) off.push_back(O[(size_t)i * n + j]);
  std::sort(off.begin(), off.end(), std::greater<double>());
  const long k = (long)keep - n;
  if (k <= 0) return 0.5 * ((off.empty() ? 0.0 : off[0]) + 1.0);
  if (k >= (long)off.size()) return 0.0;
  auto ok = [&](long j) {
    if (j < 1 || j >= (long)off.size()) return false;
    const double gap = off[j - 1] - off[j];
    return gap >= 1e-9 * 0.5 * (off[j - 1] + off[j]) && gap > 0;
  };
  long j = k;
  if (!ok(j)) {
    for (long d = 1; d < (long)off.size(); ++d) {
      if (ok(k + d)) { j = k + d; break; }
      if (ok(k - d)) { j = k - d; break; }
    }
  }
  return 0.5 * (off[j - 1] + off[j]);
}

template <typename T> T* upsi_of(bse_ctx* c);
template <> double* upsi_of<double>(bse_ctx* c) { return c->upsi64; }
template <> float* upsi_of<float>(bse_ctx* c) { return c->upsi32; }
template <typename T> T* psi_of(bse_ctx* c);
template <> double* psi_of<double>(bse_ctx* c) { return c->psi64; }
template <> float* psi_of<float>(bse_ctx* c) { return c->psi32; }
template <typename T> T* pdep_of(bse_ctx* c);
template <> double* pdep_of<double>(bse_ctx* c) { return c->pdep64; }
template <> float* pdep_of<float>(bse_ctx* c) { return c->pdep32; }
template <typename T> T* vloc_of(bse_ctx* c);
template <> double* vloc_of<double>(bse_ctx* c) { return c->vloc64; }
template <> float* vloc_of<float>(bse_ctx* c) { return c->vloc32; }
template <typename T> const T* g2h_of(bse_ctx* c);
template <> const double* g2h_of<double>(bse_ctx* c) { return c->g2h64; }
template <> const float* g2h_of<float>(bse_ctx* c) { return c->g2h32; }
template <typename T> const T* esh_of(bse_ctx* c);
template <> const double* esh_of<double>(bse_ctx* c) { return c->esh64; }
template <> const float* esh_of<float>(bse_ctx* c) { return c->esh32; }
template <typename T> const cplx<T>* tw_of(bse_ctx* c);
template <> const double2* tw_of<double>(bse_ctx* c) { return c->tw64; }
template <> const float2* tw_of<float>(bse_ctx* c) { return c->tw32; }

// ---------------------------------------------------------------------------------
// P_c = 1 - sum_v |psi_v><psi_v| on `rows` packed orbital rows (Section 2)
// ---------------------------------------------------------------------------------
template <typename T>
int project(bse_ctx* c, long rows, T* X, T* cbuf) {
  if (rows <= 0) return BSE_OK;
  if constexpr (sizeof(T) == 4) {
    if (c->tc_ok) {
      // C = X Psi^T (BF16x3 tensor cores), X -= C Psi
      CA(tc_product(c, (const float*)X, rows, c->n_pw, c->n_pw, c->psi_s, false, (float*)cbuf, c->n_occ, 1.0, 0.0));
      if (c->n_up > 0) CK(mask_cross_channel<T>((int)rows, c->n_occ, c->n_up, cbuf, c->st));
      CA(tc_product(c, (const float*)cbuf, rows, c->n_occ, c->n_occ, c->psiT_s, true, (float*)X, c->n_pw, -1.0, 1.0));
      CK(zero_pad_column<T>((int)rows, c->n_pw, X, c->st));
      return BSE_OK;
    }
  }
  const T* psi = psi_of<T>(c);
  // cbuf [rows x n_occ] = X psi^T ; X -= cbuf psi
  CK((gemm<T, T>(false, true, (int)rows, c->n_occ, c->n_pw, 1.0, X, c->n_pw, psi, c->n_pw, 0.0,
                 cbuf, c->n_occ, 1, c->st)));
  if (c->n_up > 0) CK(mask_cross_channel<T>((int)rows, c->n_occ, c->n_up, cbuf, c->st));
  CK((gemm<T, T>(false, false, (int)rows, c->n_pw, c->n_occ, -1.0, cbuf, c->n_occ, psi, c->n_pw,
                 1.0, X, c->n_pw, 1, c->st)));
  CK(zero_pad_column<T>((int)rows, c->n_pw, X, c->st));
  return BSE_OK;
}

// ---------------------------------------------------------------------------------
// explicit QP terms of D (Eq. ham): R += sum_c psi_c delta_c <psi_c|A>, c = n_occ+1..N_QP,
// on `rows` packed orbital rows; cbuf holds rows x n_qc coefficients
// ---------------------------------------------------------------------------------
template <typename T> const T* qpsi_of(bse_ctx* c);
template <> const double* qpsi_of<double>(bse_ctx* c) { return c->qpsi64; }
template <> const float* qpsi_of<float>(bse_ctx* c) { return c->qpsi32; }

template <typename T>
int qp_correction(bse_ctx* c, long rows, const T* A, T* R, T* cbuf, bool allow_tc = true) {
  if (c->n_qc == 0 || rows <= 0) return BSE_OK;
  if constexpr (sizeof(T) == 4) {
    if (c->tc_ok && allow_tc) {
      CA(tc_product(c, (const float*)A, rows, c->n_pw, c->n_pw, c->qpsi_s, false, (float*)cbuf, c->n_qc, 1.0, 0.0));
      CK(scale_columns<T>((int)rows, c->n_qc, cbuf, c->n_qc, c->qdelta, c->st));
      CA(tc_product(c, (const float*)cbuf, rows, c->n_qc, c->n_qc, c->qpsiT_s, true, (float*)R, c->n_pw, 1.0, 1.0));
      return BSE_OK;
    }
  }
  const T* q = qpsi_of<T>(c);
  CK((gemm<T, T>(false, true, (int)rows, c->n_qc, c->n_pw, 1.0, A, c->n_pw, q, c->n_pw, 0.0, cbuf, c->n_qc, 1,
                 c->st)));
  CK(scale_columns<T>((int)rows, c->n_qc, cbuf, c->n_qc, c->qdelta, c->st));
  CK((gemm<T, T>(false, false, (int)rows, c->n_pw, c->n_qc, 1.0, cbuf, c->n_qc, q, c->n_pw, 1.0, R, c->n_pw, 1,
                 c->st)));
  return BSE_OK;
}

// - sum_{w != v} E_vw a_sw for every vector s of a block (the occupied energies of Eq. d in a
// rotated frame, Eq. wannier)
template <typename T> const T* eoff_of(bse_ctx* c);
template <> const double* eoff_of<double>(bse_ctx* c) { return c->eoff64; }
template <> const float* eoff_of<float>(bse_ctx* c) { return c->eoff32; }

template <typename T>
int emat_term(bse_ctx* c, long n_vec, const T* A, T* R) {
  if (!c->has_emat) return BSE_OK;
  const long blk = (long)c->n_occ * c->n_pw;
  for (long s = 0; s < n_vec; ++s)
    CK((gemm<T, T>(false, false, c->n_occ, c->n_pw, c->n_occ, -1.0, eoff_of<T>(c), c->n_occ, A + s * blk, c->n_pw,
                   1.0, R + s * blk, c->n_pw, 1, c->st)));
  return BSE_OK;
}

// ---------------------------------------------------------------------------------
// operator workspace
// ---------------------------------------------------------------------------------
template <typename T>
int ensure_workspace(bse_ctx* c, long n_vec) {
  const size_t per_vec = (size_t)2 * ((c->n_occ + 1) / 2) * c->n3 * sizeof(cplx<T>);
  long cap = (long)std::max<size_t>(1, c->ws_budget / std::max<size_t>(1, per_vec));
  long want = std::min(n_vec, cap);
  if (want <= c->ws_vecs) return BSE_OK;
  dfree(c, c->ws_a); dfree(c, c->ws_r); dfree(c, c->ws_h); dfree(c, c->ws_c);
  c->ws_a = c->ws_r = c->ws_h = c->ws_c = nullptr;
  c->ws_vecs = 0;
  const long nf = want * c->n_occ;
  const long ngr = (nf + 1) / 2;
  cplx<T>* p;
  CA(dalloc(c, &p, (size_t)ngr * c->n3)); c->ws_a = p;
  CA(dalloc(c, &p, (size_t)ngr * c->n3)); c->ws_r = p;
  CA(dalloc(c, &p, (size_t)((want + 1) / 2) * c->n3)); c->ws_h = p;
  T* q;
  CA(dalloc(c, &q, (size_t)nf * std::max(c->n_occ, c->n_qc))); c->ws_c = q;
  c->ws_vecs = want;
  return BSE_OK;
}

// K1d variant for a block of nv vectors without tuning: the forced one, else the tuned one
// for this width, else the default
template <typename T>
int k1d_variant_for(const bse_ctx* c, int nv) {
  if (c->k1d_force) return c->k1d_force;
  auto it = c->k1d_var.find(nv);
  return it != c->k1d_var.end() ? it->second : k1d_default_variant<T>(c->n_occ, nv);
}

// ---------------------------------------------------------------------------------
// K1d tile autotuner: at the first application of a block width n_vec, time the tile
// variants (points and vectors per CTA) that fit shared memory and pad that width least
// (at most 3 padded vectors beyond the best), on the real inputs restricted to the first
// eighth of the grid points (twice each, CUDA events on the context stream), and keep the
// fastest for that width. The choice only changes the tiling, never the summation order.
// ---------------------------------------------------------------------------------
// Tuning results are shared by every context of the process with the same shape (precision,
// grid, orbital count, row-block entries, block width): a later context of the same system
// starts with the tuned variants.
std::mutex g_k1d_tune_mu;
std::map<std::tuple<int, long, int, long, int>, int> g_k1d_tuned;

template <typename T>
int autotune_k1d(bse_ctx* c, int nv, long n3, const T* ga, const T* gh, T* gr, double sf) {
  if (!c->autotune) { c->k1d_var[nv] = k1d_default_variant<T>(c->n_occ, nv); return BSE_OK; }
  const auto key = std::make_tuple((int)sizeof(T), n3, c->n_occ, (long)c->n_ent, nv);
  {
    std::lock_guard<std::mutex> lk(g_k1d_tune_mu);
    auto it = g_k1d_tuned.find(key);
    if (it != g_k1d_tuned.end()) { c->k1d_var[nv] = it->second; return BSE_OK; }
  }
  const long n_pts = std::max<long>(TAU_TB, (n3 / 8) / TAU_TB * TAU_TB);
  int least = 1 << 30;
  for (int v = 1; v <= k1d_num_variants(); ++v)
    if (k1d_fits<T>(c->n_occ, v)) least = std::min(least, k1d_padded_vectors(nv, v));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_v = 0;
  for (int v = 1; v <= k1d_num_variants(); ++v) {
    if (!k1d_fits<T>(c->n_occ, v) || k1d_padded_vectors(nv, v) > least + 3) continue;
    // one cold run, then the fastest of three timed runs
    float t = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
      CK(cudaEventRecord(e0, c->st));
      CK(k1d_tiled<T>(nv, c->n_occ, n3, ga, (const T*)c->tau, c->n_ent, c->bptr, c->bw, c->n_rblocks,
                      vloc_of<T>(c), gh, upsi_of<T>(c), sf, gr, v, c->st, n_pts));
      CK(cudaEventRecord(e1, c->st));
      CK(cudaEventSynchronize(e1));
      float tr = 0;
      CK(cudaEventElapsedTime(&tr, e0, e1));
      if (rep > 0) t = std::min(t, tr);
    }
    if (t < best) { best = t; best_v = v; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->k1d_var[nv] = best_v ? best_v : k1d_default_variant<T>(c->n_occ, nv);
  std::lock_guard<std::mutex> lk(g_k1d_tune_mu);
  g_k1d_tuned[key] = c->k1d_var[nv];
  return BSE_OK;
}

// the same tuning for the symmetric-layout kernel (its own variant list)
std::map<std::tuple<int, long, int, long, int>, int> g_k1d_sym_tuned;
K1dLists k1d_sym_lists(const bse_ctx* c);

template <typename T>
int k1d_sym_variant_for(const bse_ctx* c, int nv) {
  if (c->k1d_force_sym) return c->k1d_force_sym;
  auto it = c->k1d_var_sym.find(nv);
  return it != c->k1d_var_sym.end() ? it->second : k1d_sym_default_variant<T>(c->n_occ, nv);
}

template <typename T>
int autotune_k1d_sym(bse_ctx* c, int nv, long n3, const T* ga, const T* gh, T* gr, double sf) {
  if (!c->autotune) { c->k1d_var_sym[nv] = k1d_sym_default_variant<T>(c->n_occ, nv); return BSE_OK; }
  const auto key = std::make_tuple((int)sizeof(T), n3, c->n_occ, (long)c->n_ent_u, nv);
  {
    std::lock_guard<std::mutex> lk(g_k1d_tune_mu);
    auto it = g_k1d_sym_tuned.find(key);
    if (it != g_k1d_sym_tuned.end()) { c->k1d_var_sym[nv] = it->second; return BSE_OK; }
  }
  const long n_pts = std::max<long>(TAU_TB, (n3 / 8) / TAU_TB * TAU_TB);
  int least = 1 << 30;
  for (int v = 1; v <= k1d_sym_num_variants(); ++v)
    if (k1d_sym_fits<T>(c->n_occ, v)) least = std::min(least, k1d_sym_padded_vectors(nv, v));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_v = 0;
  const K1dLists L = k1d_sym_lists(c);
  for (int v = 1; v <= k1d_sym_num_variants(); ++v) {
    if (!k1d_sym_fits<T>(c->n_occ, v) || k1d_sym_padded_vectors(nv, v) > least + 3) continue;
    // one cold run, then the fastest of three timed runs
    float t = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
      CK(cudaEventRecord(e0, c->st));
      CK(k1d_sym_tiled<T>(nv, c->n_occ, n3, ga, (const T*)c->tau, L, vloc_of<T>(c), gh, upsi_of<T>(c), sf, gr, v,
                          c->st, n_pts));
      CK(cudaEventRecord(e1, c->st));
      CK(cudaEventSynchronize(e1));
      float tr = 0;
      CK(cudaEventElapsedTime(&tr, e0, e1));
      if (rep > 0) t = std::min(t, tr);
    }
    if (t < best) { best = t; best_v = v; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->k1d_var_sym[nv] = best_v ? best_v : k1d_sym_default_variant<T>(c->n_occ, nv);
  std::lock_guard<std::mutex> lk(g_k1d_tune_mu);
  g_k1d_sym_tuned[key] = c->k1d_var_sym[nv];
  return BSE_OK;
}

// ---------------------------------------------------------------------------------
// R = P_c (D + K1e - K1d) A   (Eqs. evp, d, k1e, k1d)
// ---------------------------------------------------------------------------------
template <typename T>
int apply_impl(bse_ctx* c, long n_vec, const T* a_in, T* a_out) {
  if (n_vec <= 0) return BSE_OK;
  CA(ensure_workspace<T>(c, n_vec));
  const long chunk = c->ws_vecs;
  const int N = c->N;
  const long n3 = c->n3;
  const T* tau = (const T*)c->tau;
  const double sf = c->k1e_factor();
  for (long s0 = 0; s0 < n_vec; s0 += chunk) {
    const long nv = std::min(chunk, n_vec - s0);
    const long nf = nv * c->n_occ;
    const long ngr = (nf + 1) / 2;
    const T* ain = a_in + s0 * c->n_occ * c->n_pw;
    T* aout = a_out + s0 * c->n_occ * c->n_pw;
    cplx<T>* ga = (cplx<T>*)c->ws_a;
    cplx<T>* gr = (cplx<T>*)c->ws_r;
    cplx<T>* gh = (cplx<T>*)c->ws_h;
    const double sz = sizeof(T), gb = (double)ngr * n3 * sizeof(cplx<T>);
    // a_sv(G) -> a_sv(r)
    // a_sv(G) -> a_sv(r): pruned transform, compact stages in the (not yet used) R(r) grids
    {
      // algorithmic bytes: the sphere read and the grid written once (the compact column stage
      // in between is the transform's own traffic, not counted)
      Scope sc(c, "fft_inverse_a", (double)nf * c->n_pw * sz + gb, fft_flops(n3, ngr));
      CK(sphere_to_grid<T>(ain, nf, c->n_pw, c->n_half, N, c->sph, tw_of<T>(c), gr, ga, c->st));
    }
    // Hartree potential of the pair density sum_w psi_w a_sw (Eq. k1e)
    const long nh = (nv + 1) / 2;
    CK(cudaMemsetAsync(gh, 0, (size_t)nh * n3 * sizeof(cplx<T>), c->st));
    if (sf != 0.0) {
      {
        Scope sc(c, "hartree_density", ((double)nf + c->n_occ + nv) * n3 * sz, 2.0 * nf * n3);
        CK(hartree_density<T>((int)nv, c->n_occ, n3, (const T*)ga, upsi_of<T>(c), (T*)gh, c->st));
      }
      Scope sc(c, "hartree_potential", 6.0 * nh * n3 * sizeof(cplx<T>), 2.0 * fft_flops(n3, nh));
      CK(fft3d<T>(gh, nh, N, -1, tw_of<T>(c), c->st));
      CK(grid_coulomb<T>(gh, nh, N, c->L, c->omega, 0, 1.0 / (double)n3, c->st));
      CK(fft3d<T>(gh, nh, N, +1, tw_of<T>(c), c->st));
    }
    // real-space combination with the screened direct term (Eq. k1d)
    if (nf & 1) CK(cudaMemsetAsync(gr + (ngr - 1) * n3, 0, (size_t)n3 * sizeof(cplx<T>), c->st));
    {
      const double nnz = (double)c->nnz;
      Scope sc(c, "k1d_combine",
               ((double)c->n_pairs + 2.0 * nf + 1.0 + nv + c->n_occ) * n3 * sz,
               (2.0 * nnz * nv + 5.0 * nf) * n3);
      if (c->tau_entry) {
        if (!c->k1d_force && !c->k1d_var.count((int)nv))
          CA(autotune_k1d<T>(c, (int)nv, n3, (const T*)ga, (const T*)gh, (T*)gr, sf));
        CK(k1d_tiled<T>((int)nv, c->n_occ, n3, (const T*)ga, tau, c->n_ent, c->bptr, c->bw, c->n_rblocks,
                        vloc_of<T>(c), (const T*)gh, upsi_of<T>(c), sf, (T*)gr, k1d_variant_for<T>(c, (int)nv),
                        c->st));
      } else if (c->tau_sym) {
        if (!c->k1d_force_sym && !c->k1d_var_sym.count((int)nv))
          CA(autotune_k1d_sym<T>(c, (int)nv, n3, (const T*)ga, (const T*)gh, (T*)gr, sf));
        CK(k1d_sym_tiled<T>((int)nv, c->n_occ, n3, (const T*)ga, tau, k1d_sym_lists(c), vloc_of<T>(c),
                            (const T*)gh, upsi_of<T>(c), sf, (T*)gr, k1d_sym_variant_for<T>(c, (int)nv), c->st));
      } else {
        CK(k1d_combine<T>((int)nv, c->n_occ, n3, (const T*)ga, tau, c->n_pairs, c->nbr_ptr, c->nbr_w, c->nbr_p,
                          vloc_of<T>(c), (const T*)gh, upsi_of<T>(c), sf, (T*)gr, c->st));
      }
    }
    // back to the sphere, plus (1/2|G|^2 + Delta - eps_v) a (Eq. d)
    // back to the sphere, plus (1/2|G|^2 + Delta - eps_v) a (Eq. d); compact stages in
    // the a(r) grids, which K1d no longer needs
    {
      // algorithmic bytes: the grid read once, the sphere written once and a(G) read once for the
      // fused diagonal term
      Scope sc(c, "fft_forward_r", gb + 2.0 * nf * c->n_pw * sz, fft_flops(n3, ngr));
      CK(grid_to_sphere<T>(gr, nf, c->n_pw, c->n_half, N, c->sph, tw_of<T>(c), ga, 1.0 / (double)n3, aout,
                           ain, g2h_of<T>(c), esh_of<T>(c), c->n_occ, c->st));
    }
    if (c->n_qc > 0) {
      Scope sc(c, "qp_terms", (3.0 * nf * c->n_pw + (double)c->n_qc * c->n_pw) * sz,
               4.0 * nf * c->n_qc * (double)c->n_pw);
      CA(qp_correction<T>(c, nf, ain, aout, (T*)c->ws_c));
    }
    if (c->has_emat) {
      Scope sc(c, "occupied_energy_matrix", 3.0 * nf * c->n_pw * sz, 2.0 * nf * c->n_occ * (double)c->n_pw);
      CA(emat_term<T>(c, nv, ain, aout));
    }
    {
      Scope sc(c, "projector_pc", (3.0 * nf * c->n_pw + (double)c->n_occ * c->n_pw) * sz,
               4.0 * nf * c->n_occ * (double)c->n_pw);
      CA(project<T>(c, nf, aout, (T*)c->ws_c));
    }
  }
  return BSE_OK;
}

// ---------------------------------------------------------------------------------
// overlaps, pair rule and screened integrals (Eqs. overlap, tau, tau_from_tau_u, pdep)
// ---------------------------------------------------------------------------------
// serialises the tau layout decision and allocation of contexts building at the same time
std::mutex g_tau_layout_mu;

// lists of the symmetric (once per pair) tau layout; pid[v][w] = pair index or -1
int build_sym_lists(bse_ctx* c, const std::vector<std::vector<int>>& pid) {
  const int n = c->n_occ;
  const int nrb = (n + 3) / 4;
  int64_t n_ent_u = 0;
  std::vector<int2> hslot_u;
  // Row blocks of 4 consecutive orbitals. Upper entries of block b: every w >= 4b that pairs
  // with a row of b (Eq. overlap); tau_vw = tau_wv (Eq. tau), so the rows' neighbours in
  // earlier blocks are read from those blocks' entries as transposed tiles.
    std::vector<int> ubptr_h(1, 0), ubw_h;
  std::vector<int> ent_of((size_t)nrb * n, -1);   // entry index of (block, w), -1 if none
  for (int b = 0; b < nrb; ++b) {
    for (int w = 4 * b; w < n; ++w) {
      bool any = false;
      for (int i = 0; i < 4; ++i) {
        const int v = 4 * b + i;
        if (v < n && pid[v][w] >= 0) any = true;
      }
      if (any) { ent_of[(size_t)b * n + w] = (int)ubw_h.size(); ubw_h.push_back(w); }
    }
    ubptr_h.push_back((int)ubw_h.size());
  }
  std::vector<int> utptr_h(1, 0), utinfo_h;
  std::vector<int4> utent_h;
  for (int b = 0; b < nrb; ++b) {
    for (int J = 0; J < b; ++J) {
      int4 q = make_int4(-1, -1, -1, -1);
      int* qq = &q.x;
      int jm = 0;
      for (int i = 0; i < 4; ++i) {
        const int v = 4 * b + i;
        if (v >= n) continue;
        qq[i] = ent_of[(size_t)J * n + v];
        for (int j = 0; j < 4; ++j)
          if (4 * J + j < n && pid[4 * J + j][v] >= 0) jm |= 1 << j;
      }
      if (jm) { utinfo_h.push_back((J << 4) | jm); utent_h.push_back(q); }
    }
    utptr_h.push_back((int)utinfo_h.size());
  }
  n_ent_u = (int64_t)ubw_h.size();
  // entry slots of every pair v <= w: row v % 4 of entry (block of v, w); inside one block
  // also row w % 4 of entry (block, v), since that block's rows read both from their own
  // entries
  hslot_u.assign(c->n_pairs, make_int2(-1, -1));
  for (int64_t p = 0; p < c->n_pairs; ++p) {
    const int v = c->pv_h[p], w = c->pw_h[p];
    const int bv = v / 4, bw_ = w / 4;
    hslot_u[p].x = 4 * ent_of[(size_t)bv * n + w] + v % 4;
    if (bv == bw_ && v != w) hslot_u[p].y = 4 * ent_of[(size_t)bv * n + v] + w % 4;
  }
  c->n_ent_u = n_ent_u;
  dfree(c, c->ubptr); dfree(c, c->ubw); dfree(c, c->utptr); dfree(c, c->utinfo); dfree(c, c->utent); dfree(c, c->uslot);
  c->ubptr = c->ubw = c->utptr = c->utinfo = nullptr; c->utent = nullptr; c->uslot = nullptr;
  CA(dalloc(c, &c->ubptr, ubptr_h.size()));
  CA(dalloc(c, &c->ubw, std::max<size_t>(1, ubw_h.size())));
  CA(dalloc(c, &c->utptr, utptr_h.size()));
  CA(dalloc(c, &c->utinfo, std::max<size_t>(1, utinfo_h.size())));
  CA(dalloc(c, &c->utent, std::max<size_t>(1, utent_h.size())));
  CA(dalloc(c, &c->uslot, hslot_u.size()));
  CK(cudaMemcpyAsync(c->ubptr, ubptr_h.data(), sizeof(int) * ubptr_h.size(), cudaMemcpyHostToDevice, c->st));
  if (!ubw_h.empty()) CK(cudaMemcpyAsync(c->ubw, ubw_h.data(), sizeof(int) * ubw_h.size(), cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->utptr, utptr_h.data(), sizeof(int) * utptr_h.size(), cudaMemcpyHostToDevice, c->st));
  if (!utinfo_h.empty()) {
    CK(cudaMemcpyAsync(c->utinfo, utinfo_h.data(), sizeof(int) * utinfo_h.size(), cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(c->utent, utent_h.data(), sizeof(int4) * utent_h.size(), cudaMemcpyHostToDevice, c->st));
  }
  CK(cudaMemcpyAsync(c->uslot, hslot_u.data(), sizeof(int2) * hslot_u.size(), cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  return BSE_OK;
}

K1dLists k1d_sym_lists(const bse_ctx* c) {
  K1dLists L;
  L.n_ent = (long)c->n_ent_u;
  L.n_blocks = c->n_rblocks;
  L.bptr = c->ubptr; L.bw = c->ubw; L.tptr = c->utptr; L.tinfo = c->utinfo; L.tent = c->utent;
  return L;
}

template <typename T>
int build_tau_impl(bse_ctx* c) {
  const long n3 = c->n3;
  const int n = c->n_occ;
  // O_vw in FP64 always, so that the lists do not depend on the precision mode
  {
    // the Gram of the densities |psi_v|^2 (FP64 values, split into FP32 hi / lo) in
    // float-float arithmetic
    float *rho_hi, *rho_lo;
    double *gram, *dg;
    CA(dalloc(c, &rho_hi, (size_t)n * n3));
    CA(dalloc(c, &rho_lo, (size_t)n * n3));
    CA(dalloc(c, &gram, (size_t)n * n));
    CA(dalloc(c, &dg, (size_t)n));
    CK(square_fields_split(n, c->upsi64, n3, rho_hi, rho_lo, c->st));
    CK(gram_ff(n, n3, rho_hi, rho_lo, n3, gram, n, c->st));
    CK(normalize_overlap(n, gram, dg, c->st));
    c->O_h.assign((size_t)n * n, 0.0);
    CK(cudaMemcpyAsync(c->O_h.data(), gram, sizeof(double) * n * n, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    dfree(c, rho_hi); dfree(c, rho_lo); dfree(c, gram); dfree(c, dg);
  }
  if (!all_finite(c->O_h.data(), (long)n * n)) return fail(c, BSE_ERR_NUMERIC, "non-finite overlap");
  // the screened direct term conserves spin: pairs across the channels of a spin-polarised
  // system are never kept and take no part in the threshold rule (overlap -1, below [0, 1])
  std::vector<double> O_rule = c->O_h;
  for (int v = 0; v < n; ++v)
    for (int w = 0; w < n; ++w)
      if (c->chan(v) != c->chan(w)) O_rule[(size_t)v * n + w] = -1.0;
  c->thr = choose_threshold(O_rule, n, c->thr_in, c->keep_pairs);
  // pair list v <= w (row-major) and CSR neighbour lists in both directions
  std::vector<std::vector<int>> pid(n, std::vector<int>(n, -1));
  c->pv_h.clear(); c->pw_h.clear();
  for (int v = 0; v < n; ++v)
    for (int w = v; w < n; ++w) {
      const bool keep = (v == w) || (O_rule[(size_t)v * n + w] >= c->thr);
      if (keep) {
        pid[v][w] = pid[w][v] = (int)c->pv_h.size();
        c->pv_h.push_back(v); c->pw_h.push_back(w);
      }
    }
  c->n_pairs = (int64_t)c->pv_h.size();
  std::vector<int> ptr(n + 1, 0), nw, np;
  for (int v = 0; v < n; ++v) {
    for (int w = 0; w < n; ++w)
      if (pid[v][w] >= 0) { nw.push_back(w); np.push_back(pid[v][w]); }
    ptr[v + 1] = (int)nw.size();
  }
  c->nnz = (int64_t)nw.size();
  // block-CSR over row blocks of 4 consecutive orbitals
  std::vector<int> hbptr(1, 0), hbw;
  std::vector<int4> hbp;
  const int nrb = (n + 3) / 4;
  for (int b = 0; b < nrb; ++b) {
    for (int w = 0; w < n; ++w) {
      int4 q; q.x = q.y = q.z = q.w = -1;
      bool any = false;
      int* qq = &q.x;
      for (int i = 0; i < 4; ++i) {
        const int v = 4 * b + i;
        if (v < n && pid[v][w] >= 0) { qq[i] = pid[v][w]; any = true; }
      }
      if (any) { hbw.push_back(w); hbp.push_back(q); }
    }
    hbptr.push_back((int)hbw.size());
  }
  c->n_rblocks = nrb;
  c->n_ent = (int64_t)hbw.size();
  // entry slots of every pair: (v, w) sits in row v % 4 of entry (block of v, w) and, for
  // v != w, in row w % 4 of entry (block of w, v)
  std::vector<int2> hslot(c->n_pairs, make_int2(-1, -1));
  for (int b = 0; b < nrb; ++b)
    for (int e = hbptr[b]; e < hbptr[b + 1]; ++e) {
      const int* qq = &hbp[e].x;
      for (int i = 0; i < 4; ++i) {
        const int p = qq[i];
        if (p < 0) continue;
        if (hslot[p].x < 0) hslot[p].x = 4 * e + i;
        else hslot[p].y = 4 * e + i;
      }
    }
  dfree(c, c->nbr_ptr); dfree(c, c->nbr_w); dfree(c, c->nbr_p); dfree(c, c->pv); dfree(c, c->pw);
  dfree(c, c->tau); c->tau = nullptr;
  CA(dalloc(c, &c->nbr_ptr, ptr.size()));
  CA(dalloc(c, &c->nbr_w, nw.size()));
  CA(dalloc(c, &c->nbr_p, np.size()));
  dfree(c, c->bptr); dfree(c, c->bw); dfree(c, c->tslot);
  CA(dalloc(c, &c->bptr, hbptr.size()));
  CA(dalloc(c, &c->bw, std::max<size_t>(1, hbw.size())));
  CA(dalloc(c, &c->tslot, hslot.size()));
  CK(cudaMemcpyAsync(c->bptr, hbptr.data(), sizeof(int) * hbptr.size(), cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->bw, hbw.data(), sizeof(int) * hbw.size(), cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->tslot, hslot.data(), sizeof(int2) * hslot.size(), cudaMemcpyHostToDevice, c->st));
  CA(dalloc(c, &c->pv, c->pv_h.size()));
  CA(dalloc(c, &c->pw, c->pw_h.size()));
  CK(cudaMemcpyAsync(c->nbr_ptr, ptr.data(), sizeof(int) * ptr.size(), cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->nbr_w, nw.data(), sizeof(int) * nw.size(), cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->nbr_p, np.data(), sizeof(int) * np.size(), cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->pv, c->pv_h.data(), sizeof(int) * c->pv_h.size(), cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->pw, c->pw_h.data(), sizeof(int) * c->pw_h.size(), cudaMemcpyHostToDevice, c->st));
  // tau_vw = v^{1/2} (1 + chi_bar) v^{1/2} (psi_v psi_w), batched over pairs
  // the tiled K1d kernel reads tau entry-major (four rows per entry, zeros where a row lacks
  // the neighbour); the untiled fallback reads it per pair. The entry-major layout holds
  // about 2.8 times the per-pair values, so it is used only while it takes at most half of
  // the free device memory (large FP64 systems keep the per-pair layout);
  // BSE_TAU_LAYOUT=pair forces the per-pair layout and the untiled kernel.
  // Layout: the ordered entry-major tau where it takes at most half of the free memory, else
  // the symmetric one (each pair once) where that fits, else the per-pair layout with the
  // untiled kernel; BSE_TAU_LAYOUT=upper or pair skips the earlier choices. The first build of
  // a context decides and later builds keep that layout (their free memory no longer shows
  // what the context itself holds, e.g. blocks a caching allocator keeps for it). Contexts
  // that build tau at the same time (bse_solve_batch) take the decision and the allocation
  // one after another, so each sees the memory the earlier ones took.
  T* tau;
  {
    std::lock_guard<std::mutex> lk(g_tau_layout_mu);
    size_t fr = 0, tot = 0;
    CK(cudaMemGetInfo(&fr, &tot));
    const double half = 0.5 * (double)fr;
    const char* lay = getenv("BSE_TAU_LAYOUT");
    const bool force_pair = lay && std::strcmp(lay, "pair") == 0;
    const bool force_upper = lay && std::strcmp(lay, "upper") == 0;
    const bool tiled = n3 % TAU_TB == 0;
    const double t4 = (double)c->n_ent * 4.0 * (double)n3 * sizeof(T);
    c->tau_entry = c->tau_sym = false;
    if (c->tau_layout == 1) {
      c->tau_entry = true;
    } else if (c->tau_layout == 2) {
      CA(build_sym_lists(c, pid));
      c->tau_sym = true;
    } else if (c->tau_layout < 0) {
      if (!force_pair && !force_upper && tiled && k1d_default_variant<T>(c->n_occ, 1) > 0 && t4 <= half) {
        c->tau_entry = true;
      } else if (!force_pair && tiled && k1d_sym_default_variant<T>(c->n_occ, 1) > 0) {
        CA(build_sym_lists(c, pid));
        c->tau_sym = (double)c->n_ent_u * 4.0 * (double)n3 * sizeof(T) <= half;
      }
      c->tau_layout = c->tau_entry ? 1 : (c->tau_sym ? 2 : 0);
    }
    if (c->tau_entry) {
      CA(dalloc(c, &tau, (size_t)c->n_ent * 4 * n3));
    } else if (c->tau_sym) {
      CA(dalloc(c, &tau, (size_t)c->n_ent_u * 4 * n3));
    } else {
      CA(dalloc(c, &tau, (size_t)c->n_pairs * n3));
    }
    CK(cudaStreamSynchronize(c->st));   // the allocation is visible in the next context's free memory
  }
  if (c->tau_entry) CK(cudaMemsetAsync(tau, 0, sizeof(T) * (size_t)c->n_ent * 4 * n3, c->st));
  if (c->tau_sym) CK(cudaMemsetAsync(tau, 0, sizeof(T) * (size_t)c->n_ent_u * 4 * n3, c->st));
  c->tau = tau;
  const size_t budget = (size_t)2 << 30;
  long nb = (long)(budget / (n3 * sizeof(cplx<T>))) * 2;
  nb = std::max<long>(2, std::min<long>(nb, 4096));
  nb = std::min<long>(nb, (c->n_pairs + 1) / 2 * 2);
  cplx<T>* grids;
  T *X, *X2, *Cp;
  CA(dalloc(c, &grids, (size_t)((nb + 1) / 2) * n3));
  CA(dalloc(c, &X, (size_t)nb * c->n_pw));
  CA(dalloc(c, &X2, (size_t)nb * c->n_pw));
  CA(dalloc(c, &Cp, (size_t)nb * std::max(1, c->n_pdep)));
  const T* pd = pdep_of<T>(c);
  for (long p0 = 0; p0 < c->n_pairs; p0 += nb) {
    const int b = (int)std::min<long>(nb, c->n_pairs - p0);
    const long ng = (b + 1) / 2;
    const double gbt = (double)ng * n3 * sizeof(cplx<T>);
    Scope sc(c, "tau_build", gbt * 8.0 + (double)b * n3 * sizeof(T),
             2.0 * fft_flops(n3, ng) + 4.0 * b * (double)c->n_pdep * c->n_pw);
    CK(pair_product<T>(b, c->pv + p0, c->pw + p0, upsi_of<T>(c), n3, 1.0 / c->omega, grids, c->st));
    CK(fft3d<T>(grids, ng, c->N, -1, tw_of<T>(c), c->st));
    CK(grid_coulomb<T>(grids, ng, c->N, c->L, c->omega, 1, 1.0 / (double)n3, c->st));
    if (c->n_pdep > 0) {
      CK((sphere_pack<T, T>(grids, b, c->n_pw, c->n_half, c->gpos, c->gneg, n3, 1.0, X, nullptr,
                            nullptr, nullptr, 1, c->st)));
      bool done = false;
      if constexpr (sizeof(T) == 4) {
        if (c->tc_ok) {
          CA(tc_product(c, (const float*)X, b, c->n_pw, c->n_pw, c->pdep_s, false, (float*)Cp, c->n_pdep, 1.0, 0.0));
          CK(scale_columns<T>(b, c->n_pdep, Cp, c->n_pdep, c->f, c->st));
          CA(tc_product(c, (const float*)Cp, b, c->n_pdep, c->n_pdep, c->pdepT_s, true, (float*)X2, c->n_pw, 1.0, 0.0));
          done = true;
        }
      }
      if (!done) {
        CK((gemm<T, T>(false, true, b, c->n_pdep, c->n_pw, 1.0, X, c->n_pw, pd, c->n_pw, 0.0, Cp,
                       c->n_pdep, 1, c->st)));
        CK(scale_columns<T>(b, c->n_pdep, Cp, c->n_pdep, c->f, c->st));
        CK((gemm<T, T>(false, false, b, c->n_pw, c->n_pdep, 1.0, Cp, c->n_pdep, pd, c->n_pw, 0.0, X2,
                       c->n_pw, 1, c->st)));
      }
      CK((sphere_unpack<T, T>(X2, b, c->n_pw, c->n_half, c->gpos, c->gneg, grids, n3, false, true, c->st)));
    }
    CK(grid_coulomb<T>(grids, ng, c->N, c->L, c->omega, 1, 1.0, c->st));
    CK(fft3d<T>(grids, ng, c->N, +1, tw_of<T>(c), c->st));
    if (c->tau_entry) CK(scatter_tau4<T>(b, grids, n3, p0, c->tslot, c->n_ent, tau, c->st));
    else if (c->tau_sym) CK(scatter_tau4<T>(b, grids, n3, p0, c->uslot, c->n_ent_u, tau, c->st));
    else CK(deinterleave_pairs<T>(b, grids, n3, p0, c->n_pairs, tau, c->st));
  }
  CK(cudaStreamSynchronize(c->st));
  dfree(c, grids); dfree(c, X); dfree(c, X2); dfree(c, Cp);
  c->tau_ready = true;
  return BSE_OK;
}

// ---------------------------------------------------------------------------------
// block Davidson (Section 3); algebra in FP64 (Gram / Rayleigh-Ritz accumulate in
// FP64, Jacobi eigensolver and Cholesky in FP64), vectors in the context precision
// ---------------------------------------------------------------------------------
struct Cand { double d; long flat; };

// called each iteration with the Ritz vectors X, residuals R (device, kk rows), the Ritz
// values and the indices that receive corrections
template <typename T>
using SampleHook = std::function<int(int, const T*, const T*, const std::vector<double>&,
                                     const std::vector<int>&)>;

// C (M x N, double) = A B^T over the long dimension K: the Gram, Rayleigh-Ritz and CGS
// coefficient products of the Davidson algebra (the tall-skinny SIMT kernel for N <= 32).
// Tensor cores do not pay here: an MMA with N = 32 runs at an eighth of the pipe's rate,
// and the three-term split that FP32 accuracy needs leaves them below the FP32 SIMT rate.
template <typename T>
cudaError_t tn_product(bse_ctx* c, int M, int N, long K, const T* A, long lda, const T* B, long ldb, double* C,
                       long ldc) {
  return gemm<T, double>(false, true, M, N, (int)K, 1.0, A, lda, B, ldb, 0.0, C, ldc, 0, c->st);
}

template <typename T>
int davidson_impl(bse_ctx* c, const bse_davidson_opts* o, double* omega_out, T* vec_out,
                  bse_davidson_stats* stats, const SampleHook<T>* hook = nullptr) {
  using clk = std::chrono::steady_clock;
  const auto t_start = clk::now();
  const int ne = o->n_eig, b = o->block, ms = o->max_sub;
  const long dim = (long)c->n_occ * c->n_pw;
  if (ne < 1 || b < 1 || ms < 2 * ne + b || ms > 160 || b > 128 || o->max_it < 1 || !(o->res_tol > 0))
    return fail(c, BSE_ERR_INVALID_ARG, "davidson options: need n_eig>=1, 1<=block<=128, 2*n_eig+block<=max_sub<=160, max_it>=1, res_tol>0");
  if ((long)ne > dim) return fail(c, BSE_ERR_INVALID_ARG, "n_eig exceeds the problem dimension");
  const int keep = 2 * ne;
  std::vector<void*> mine;
  auto al = [&](auto** p, size_t n) {
    int r = dalloc(c, p, n);
    if (r == BSE_OK) mine.push_back(*p);
    return r;
  };
  struct Guard {
    bse_ctx* c; std::vector<void*>* m;
    ~Guard() { for (void* p : *m) dfree(c, p); }
  } guard{c, &mine};
  T *V, *W, *X, *LX, *Rr, *Tt, *Tt2, *S1, *S2, *Yt, *Cmt, *Lt;
  double *Hs, *Yv, *jw, *theta, *nrm, *Cm, *Sg, *Linv;
  int *info, *which;
  CA(al(&V, (size_t)ms * dim)); CA(al(&W, (size_t)ms * dim));
  CA(al(&X, (size_t)ne * dim)); CA(al(&LX, (size_t)ne * dim)); CA(al(&Rr, (size_t)ne * dim));
  CA(al(&Tt, (size_t)b * dim)); CA(al(&Tt2, (size_t)b * dim));
  CA(al(&S1, (size_t)keep * dim)); CA(al(&S2, (size_t)keep * dim));
  CA(al(&Yt, (size_t)ms * ms)); CA(al(&Cmt, (size_t)ms * b)); CA(al(&Lt, (size_t)b * b));
  CA(al(&Hs, (size_t)ms * ms)); CA(al(&Yv, (size_t)ms * ms)); CA(al(&jw, (size_t)4 * ms * ms + 2 * (size_t)ms));
  CA(al(&theta, (size_t)ms)); CA(al(&nrm, (size_t)ms)); CA(al(&Cm, (size_t)ms * b));
  CA(al(&Sg, (size_t)b * b)); CA(al(&Linv, (size_t)b * b));
  CA(al(&info, 4)); CA(al(&which, (size_t)b));
  T* pcbuf = nullptr;
  CA(al(&pcbuf, (size_t)b * c->n_occ * c->n_occ + 16));
  double ms_apply = 0;
  int n_apply = 0;
  // operator applications are timed by CUDA events on the context stream (read once the solve
  // has finished), so timing them does not stall the stream
  struct ApplyEvents {
    std::vector<cudaEvent_t> ev;
    ~ApplyEvents() { for (cudaEvent_t e : ev) cudaEventDestroy(e); }
  } apply_ev;
  auto timed_apply = [&](long nv, const T* in, T* out) -> int {
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    apply_ev.ev.push_back(e0);
    CK(cudaEventCreate(&e1));
    apply_ev.ev.push_back(e1);
    CK(cudaEventRecord(e0, c->st));
    int r = apply_impl<T>(c, nv, in, out);
    if (r != BSE_OK) return r;
    CK(cudaEventRecord(e1, c->st));
    n_apply += (int)nv;
    return BSE_OK;
  };
  auto apply_ms = [&]() {
    double t = 0;
    for (size_t i = 0; i + 1 < apply_ev.ev.size(); i += 2) {
      float ms = 0;
      if (cudaEventElapsedTime(&ms, apply_ev.ev[i], apply_ev.ev[i + 1]) == cudaSuccess) t += ms;
    }
    return t;
  };
  auto proj = [&](long nvec, T* Xp) -> int {
    // P_c row by row in chunks of `b` vectors (cbuf holds b * n_occ x n_occ)
    for (long i = 0; i < nvec; i += b) {
      const long k = std::min<long>(b, nvec - i);
      CA(project<T>(c, k * c->n_occ, Xp + i * dim, pcbuf));
    }
    return BSE_OK;
  };
  // ---- initial guess: unit vectors at the lowest diagonal entries ----
  std::vector<int> order(c->n_occ);
  for (int v = 0; v < c->n_occ; ++v) order[v] = v;
  auto dval = [&](int v, int j) { return 0.5 * c->g2p_h[j] + c->v0 + c->scissor - c->eps_h[v]; };
  // merge of the per-orbital lists (g2p_h is non-decreasing in j apart from the pad j = 1)
  std::vector<std::vector<int>> jord(1);
  {
    std::vector<int> js(c->n_pw);
    for (int j = 0; j < c->n_pw; ++j) js[j] = j;
    std::stable_sort(js.begin(), js.end(), [&](int a, int bb) { return c->g2p_h[a] < c->g2p_h[bb]; });
    jord[0] = js;
  }
  auto cmp = [](const std::pair<Cand, int>& a, const std::pair<Cand, int>& bb) {
    if (a.first.d != bb.first.d) return a.first.d > bb.first.d;
    return a.first.flat > bb.first.flat;
  };
  std::priority_queue<std::pair<Cand, int>, std::vector<std::pair<Cand, int>>, decltype(cmp)> pq(cmp);
  std::vector<int> pos(c->n_occ, 0);
  // ties within one orbital's list must come out in flat-index order: re-sort equal-d runs
  {
    auto& js = jord[0];
    std::stable_sort(js.begin(), js.end(), [&](int a, int bb) {
      if (c->g2p_h[a] != c->g2p_h[bb]) return c->g2p_h[a] < c->g2p_h[bb];
      return a < bb;
    });
  }
  for (int v = 0; v < c->n_occ; ++v) {
    const int j = jord[0][0];
    pq.push({Cand{dval(v, j), (long)v * c->n_pw + j}, v});
  }
  int m = 0;
  std::vector<double> hn(std::max(ms, b));
  while (m < b && !pq.empty()) {
    auto top = pq.top(); pq.pop();
    const int v = top.second;
    if (++pos[v] < c->n_pw) {
      const int j = jord[0][pos[v]];
      pq.push({Cand{dval(v, j), (long)v * c->n_pw + j}, v});
    }
    // P_c acts on each orbital row alike, so (for the orthonormal orbitals the interface
    // requires) the projected unit vector at coordinate j keeps 1 - sum_w psi_w(j)^2 of its
    // squared norm in every row; orthogonalising against
    // accepted vectors only lowers it. A candidate below the acceptance norm (0.1) by a
    // margin beyond rounding, or at the pad coordinate, is rejected without device work.
    {
      const int jc = (int)(top.first.flat % c->n_pw);
      if (jc == 1 || 1.0 - c->occw_h[(size_t)c->chan(v) * c->n_pw + jc] < 0.01 * (1.0 - 1e-3)) continue;
    }
    T* x = V + (long)m * dim;
    CK(set_unit<T>(x, dim, top.first.flat, c->st));
    CA(project<T>(c, c->n_occ, x, pcbuf));
    for (int pass = 0; pass < 2 && m > 0; ++pass) {
      CK(tn_product<T>(c, m, 1, dim, V, dim, x, dim, Cm, 1));
      CK((convert<double, T>(m, Cm, Cmt, c->st)));
      CK((gemm<T, T>(true, false, 1, (int)dim, m, -1.0, Cmt, 1, V, dim, 1.0, x, dim, 1, c->st)));
    }
    CK(row_norms2<T>(1, dim, x, nrm, c->st));
    double n2 = 0;
    CK(cudaMemcpyAsync(&n2, nrm, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    if (std::sqrt(n2) > 0.1) {
      const double s = 1.0 / std::sqrt(n2);
      CK(cudaMemcpyAsync(nrm, &s, sizeof(double), cudaMemcpyHostToDevice, c->st));
      CK(scale_rows<T>(1, dim, x, nrm, c->st));
      ++m;
    }
  }
  if (m == 0) return fail(c, BSE_ERR_NUMERIC, "no initial vector survives the projection");
  CA(timed_apply(m, V, W));
  // Rayleigh-Ritz matrix Hs = V W^T kept with leading dimension ms and updated by columns
  {
    Scope sc(c, "davidson_rr", 2.0 * m * (double)dim * sizeof(T), 2.0 * m * m * (double)dim);
    CK(tn_product<T>(c, m, m, dim, V, dim, W, dim, Hs, ms));
    CK(symmetrize(m, Hs, ms, c->st));
  }
  int it = 0;
  bool converged = false;
  std::vector<double> th(ms), rn(ms);
  int kk = 0;
  bool use_learned = (o->precond == 1) && c->lp_params != nullptr;
  int fallbacks = (o->precond == 1 && c->lp_params == nullptr) ? 1 : 0;
  std::vector<double> res_hist;
  while (true) {
    ++it;
    // the k lowest Ritz pairs are all the algebra needs: n_eig for the residuals and
    // 2 n_eig for a restart; Yv is m x ky row-major
    const int ky = std::min(m, keep);
    {
      Scope sc(c, "davidson_eigh", 8.0 * m * m, 4.0 / 3.0 * m * m * (double)m);
      CK(eigh_lowest(m, ky, Hs, ms, jw, Yv, theta, info, sizeof(T) == 4, c->st));
    }
    kk = std::min(ne, m);
    {
      Scope sc(c, "davidson_ritz", 2.0 * (2.0 * m + 3.0 * kk) * (double)dim * sizeof(T),
               4.0 * kk * m * (double)dim);
      CK((convert<double, T>((long)m * ky, Yv, Yt, c->st)));
      CK((gemm<T, T>(true, false, kk, (int)dim, m, 1.0, Yt, ky, V, dim, 0.0, X, dim, 1, c->st)));
      CK((gemm<T, T>(true, false, kk, (int)dim, m, 1.0, Yt, ky, W, dim, 0.0, LX, dim, 1, c->st)));
      CK(residuals<T>(kk, dim, X, LX, theta, Rr, nrm, c->st));
    }
    CK(cudaMemcpyAsync(th.data(), theta, sizeof(double) * kk, cudaMemcpyDeviceToHost, c->st));
    CK(cudaMemcpyAsync(rn.data(), nrm, sizeof(double) * kk, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    if (!all_finite(th.data(), kk) || !all_finite(rn.data(), kk))
      return fail(c, BSE_ERR_NUMERIC, "non-finite Ritz value or residual");
    std::vector<int> todo;
    for (int i = 0; i < kk; ++i) {
      rn[i] = std::sqrt(rn[i]);
      if (rn[i] > o->res_tol && (int)todo.size() < b) todo.push_back(i);
    }
    if (hook && !todo.empty()) CA((*hook)(kk, X, Rr, th, todo));
    if (kk == ne && todo.empty()) { converged = true; break; }
    if (it >= o->max_it) break;
    int nt = (int)todo.size();
    if (nt == 0) break;
    CK(cudaMemcpyAsync(which, todo.data(), sizeof(int) * nt, cudaMemcpyHostToDevice, c->st));
    // learned preconditioner with the diagonal one as fallback: on a non-finite output,
    // and for good once the residuals stagnate (no 1% gain of the largest residual over
    // eight iterations)
    {
      double rmax = 0;
      for (int i = 0; i < kk; ++i) rmax = std::max(rmax, rn[i]);
      res_hist.push_back(rmax);
      if (use_learned && res_hist.size() > 8) {
        double before = 1e300, recent = 1e300;
        for (size_t q = 0; q + 8 < res_hist.size(); ++q) before = std::min(before, res_hist[q]);
        for (size_t q = res_hist.size() - 8; q < res_hist.size(); ++q) recent = std::min(recent, res_hist[q]);
        if (recent > 0.99 * before) { use_learned = false; ++fallbacks; }
      }
    }
    {
      Scope sc(c, "davidson_precond", 2.0 * nt * (double)dim * sizeof(T), 4.0 * nt * c->n_occ * (double)dim);
      bool diag = !use_learned;
      if (use_learned) {
        CK(cudaMemsetAsync(c->d_bad, 0, sizeof(int), c->st));
        CK(precond_learned<T>(nt, c->n_occ, c->n_pw, c->lp_params, Rr, theta, nrm, which, c->g2p,
                              c->eps, c->v0, c->scissor, Tt, c->d_bad, c->st));
        int hb = 0;
        CK(cudaMemcpyAsync(&hb, c->d_bad, sizeof(int), cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        if (hb) { diag = true; ++fallbacks; }
      }
      if (diag)
        CK(precond_diag<T>(nt, c->n_occ, c->n_pw, Rr, theta, which, g2h_of<T>(c), c->eps, c->v0, c->scissor,
                           Tt, c->st));
      CA(proj(nt, Tt));
    }
    if (m + nt > ms) {
      const int kp = std::min(keep, m);
      CK((gemm<T, T>(true, false, kp, (int)dim, m, 1.0, Yt, ky, V, dim, 0.0, S1, dim, 1, c->st)));
      CK((gemm<T, T>(true, false, kp, (int)dim, m, 1.0, Yt, ky, W, dim, 0.0, S2, dim, 1, c->st)));
      CK(cudaMemcpyAsync(V, S1, sizeof(T) * kp * dim, cudaMemcpyDeviceToDevice, c->st));
      CK(cudaMemcpyAsync(W, S2, sizeof(T) * kp * dim, cudaMemcpyDeviceToDevice, c->st));
      m = kp;
      Scope sc(c, "davidson_rr", 2.0 * m * (double)dim * sizeof(T), 2.0 * m * m * (double)dim);
      CK(tn_product<T>(c, m, m, dim, V, dim, W, dim, Hs, ms));
      CK(symmetrize(m, Hs, ms, c->st));
    }
    // CGS2 against V, dropping directions that lose all but 1e-8 of their norm
    std::unique_ptr<Scope> sc_orth(new Scope(c, "davidson_orth", (4.0 * m + 8.0 * nt) * (double)dim * sizeof(T),
                                             8.0 * m * nt * (double)dim + 4.0 * nt * nt * (double)dim));
    std::vector<double> n0(nt), n1(nt);
    CK(row_norms2<T>(nt, dim, Tt, nrm, c->st));
    CK(cudaMemcpyAsync(n0.data(), nrm, sizeof(double) * nt, cudaMemcpyDeviceToHost, c->st));
    // second pass only where the first removed more than half of a direction's squared
    // norm (the Daniel-Gragg-Kaufman-Stewart test with eta = 1/sqrt 2): without that much
    // cancellation one pass already leaves the rounding level of the data
    bool cancelled = false;
    for (int pass = 0; pass < 2; ++pass) {
      CK(tn_product<T>(c, m, nt, dim, V, dim, Tt, dim, Cm, nt));
      CK((convert<double, T>((long)m * nt, Cm, Cmt, c->st)));
      CK((gemm<T, T>(true, false, nt, (int)dim, m, -1.0, Cmt, nt, V, dim, 1.0, Tt, dim, 1, c->st)));
      CK(row_norms2<T>(nt, dim, Tt, nrm, c->st));
      CK(cudaMemcpyAsync(n1.data(), nrm, sizeof(double) * nt, cudaMemcpyDeviceToHost, c->st));
      CK(cudaStreamSynchronize(c->st));
      if (pass == 0) {
        for (int t = 0; t < nt; ++t)
          if (n1[t] < 0.5 * n0[t]) cancelled = true;
        if (!cancelled) break;
      }
    }
    {
      // A direction that lost all but drop_tol of its norm is rounding noise of the
      // projection and orthogonalisation, not a search direction: in the mixed path the
      // BF16x3 projector leaves ~1e-5 of occupied-space leakage, so such a direction
      // would be mostly leakage after normalisation.
      const double drop_tol = (sizeof(T) == 8) ? 1e-8 : 1e-3;
      int w = 0;
      for (int t = 0; t < nt; ++t) {
        if (std::sqrt(n1[t]) > drop_tol * std::sqrt(n0[t]) && n1[t] > 0) {
          if (w != t)
            CK(cudaMemcpyAsync(Tt + (long)w * dim, Tt + (long)t * dim, sizeof(T) * dim,
                               cudaMemcpyDeviceToDevice, c->st));
          ++w;
        }
      }
      nt = w;
    }
    if (nt == 0) break;
    // mixed path: project the kept directions once more so their occupied-space leakage
    // (the BF16x3 projector's ~1e-5, carried along by the subtraction of V C) does not
    // accumulate in the basis; skipping it when no direction cancelled raised the residual
    // floor of the medium solve to the convergence tolerance
    if (sizeof(T) == 4) CA(proj(nt, Tt));
    // CholQR2 among the new directions; a failing pivot drops that direction
    for (int pass = 0; pass < 2; ++pass) {
      while (true) {
        CK(tn_product<T>(c, nt, nt, dim, Tt, dim, Tt, dim, Sg, nt));
        CK(symmetrize(nt, Sg, nt, c->st));
        CK(cholesky_inverse(nt, Sg, nt, Linv, info, c->st));
        int hinfo = 0;
        CK(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        if (hinfo == 0) break;
        const int bad = hinfo - 1;
        for (int t = bad + 1; t < nt; ++t)
          CK(cudaMemcpyAsync(Tt + (long)(t - 1) * dim, Tt + (long)t * dim, sizeof(T) * dim,
                             cudaMemcpyDeviceToDevice, c->st));
        --nt;
        if (nt == 0) break;
      }
      if (nt == 0) break;
      CK((convert<double, T>((long)nt * nt, Linv, Lt, c->st)));
      CK((gemm<T, T>(false, false, nt, (int)dim, nt, 1.0, Lt, nt, Tt, dim, 0.0, Tt2, dim, 1, c->st)));
      std::swap(Tt, Tt2);
    }
    if (nt == 0) break;
    sc_orth.reset();
    CK(cudaMemcpyAsync(V + (long)m * dim, Tt, sizeof(T) * nt * dim, cudaMemcpyDeviceToDevice, c->st));
    CA(timed_apply(nt, V + (long)m * dim, W + (long)m * dim));
    {
      Scope sc(c, "davidson_rr", (m + 2.0 * nt) * (double)dim * sizeof(T),
               2.0 * (m + nt) * nt * (double)dim);
      CK(tn_product<T>(c, m + nt, nt, dim, V, dim, W + (long)m * dim, dim, Hs + m, ms));
      CK(mirror_new(Hs, ms, m, m + nt, c->st));
    }
    m += nt;
  }
  for (int i = 0; i < ne; ++i) omega_out[i] = i < kk ? th[i] : NAN;
  if (vec_out) CK(cudaMemcpyAsync(vec_out, X, sizeof(T) * (size_t)kk * dim, cudaMemcpyDeviceToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (stats) {
    stats->iterations = it;
    stats->n_apply = n_apply;
    ms_apply = apply_ms();
    stats->ms_apply = ms_apply;
    stats->ms_total = std::chrono::duration<double, std::milli>(clk::now() - t_start).count();
    double mx = 0;
    for (int i = 0; i < kk; ++i) mx = std::max(mx, rn[i]);
    stats->res_max = mx;
    stats->precond_fallbacks = fallbacks;
  }
  if (!converged) return fail(c, BSE_ERR_NOT_CONVERGED, "Davidson did not converge within max_it");
  return BSE_OK;
}

// ---------------------------------------------------------------------------------
// Lanczos chains for the absorption spectrum (Section 4: N_Lanczos applications of the
// operator per polarisation direction). All directions run together as one block; the
// three-term recursion stays on the device, so the chain needs no host round trip.
// ---------------------------------------------------------------------------------
template <typename T>
int lanczos_impl(bse_ctx* c, int np, const int* dirs, int m, double* alpha_h, double* beta_h, double* norm2_h) {
  const long dim = (long)c->n_occ * c->n_pw;
  std::vector<void*> mine;
  auto al = [&](auto** p, size_t n) {
    int r = dalloc(c, p, n);
    if (r == BSE_OK) mine.push_back(*p);
    return r;
  };
  struct Guard {
    bse_ctx* c; std::vector<void*>* m;
    ~Guard() { for (void* p : *m) dfree(c, p); }
  } guard{c, &mine};
  T *Q, *Qp, *W, *pcbuf;
  double *gd, *n2, *C, *alpha, *beta, *b0;
  CA(al(&Q, (size_t)np * dim)); CA(al(&Qp, (size_t)np * dim)); CA(al(&W, (size_t)np * dim));
  CA(al(&pcbuf, (size_t)np * c->n_occ * c->n_occ + 16));
  CA(al(&gd, (size_t)np * c->n_pw)); CA(al(&n2, (size_t)np)); CA(al(&C, (size_t)np * np));
  CA(al(&alpha, (size_t)np * m)); CA(al(&beta, (size_t)np * m)); CA(al(&b0, (size_t)np));
  std::vector<double> gh((size_t)np * c->n_pw);
  for (int p = 0; p < np; ++p)
    std::copy(c->gcart_h.begin() + (size_t)dirs[p] * c->n_pw, c->gcart_h.begin() + (size_t)(dirs[p] + 1) * c->n_pw,
              gh.begin() + (size_t)p * c->n_pw);
  CK(cudaMemcpyAsync(gd, gh.data(), sizeof(double) * gh.size(), cudaMemcpyHostToDevice, c->st));
  CK(cudaMemsetAsync(alpha, 0, sizeof(double) * np * m, c->st));
  CK(cudaMemsetAsync(beta, 0, sizeof(double) * np * m, c->st));
  // start block d = P_c(-d psi / d r_i), then q_1 = d / |d|
  for (int p = 0; p < np; ++p) CK(dipole_rhs<T>(c->n_occ, c->n_pw, c->psi64, gd + (size_t)p * c->n_pw, W + p * dim, c->st));
  CA(project<T>(c, (long)np * c->n_occ, W, pcbuf));
  CK(row_norms2<T>(np, dim, W, n2, c->st));
  CK(cudaMemcpyAsync(norm2_h, n2, sizeof(double) * np, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  for (int p = 0; p < np; ++p)
    if (!(norm2_h[p] > 0) || !std::isfinite(norm2_h[p]))
      return fail(c, BSE_ERR_NUMERIC, "the dipole start vector vanishes in the conduction space");
  CK(lanczos_normalize<T>(np, dim, W, n2, Q, b0, 1, c->st));
  CK(cudaMemsetAsync(Qp, 0, sizeof(T) * np * dim, c->st));
  for (int k = 0; k < m; ++k) {
    CA(apply_impl<T>(c, np, Q, W));                                              // w = L q_k
    if (k > 0) CK(lanczos_axpy<T>(np, dim, W, Qp, beta + k, m, nullptr, 0, c->st));   // - beta_k q_{k-1}
    {
      Scope sc(c, "lanczos_recursion", 4.0 * np * (double)dim * sizeof(T), 6.0 * np * (double)dim);
      CK(tn_product<T>(c, np, np, dim, Q, dim, W, dim, C, np));                 // alpha_k = <q_k|w>
      CK(lanczos_axpy<T>(np, dim, W, Q, C, np + 1, alpha + k, m, c->st));       // w -= alpha_k q_k
      if (k + 1 < m) {
        // back onto the conduction space: rounding components in the occupied space (where L
        // is zero) would grow exponentially under the three-term recurrence
        CA(project<T>(c, (long)np * c->n_occ, W, pcbuf));
        CK(row_norms2<T>(np, dim, W, n2, c->st));                               // beta_{k+1} = |w|
        std::swap(Q, Qp);
        CK(lanczos_normalize<T>(np, dim, W, n2, Q, beta + k + 1, m, c->st));    // q_{k+1} = w / beta
      }
    }
  }
  CK(cudaMemcpyAsync(alpha_h, alpha, sizeof(double) * np * m, cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(beta_h, beta, sizeof(double) * np * m, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (!all_finite(alpha_h, (long)np * m) || !all_finite(beta_h, (long)np * m))
    return fail(c, BSE_ERR_NUMERIC, "non-finite Lanczos coefficient");
  return BSE_OK;
}

int spectrum_impl(bse_ctx* c, int m, const double* alpha_h, const double* beta_h, double norm2, int n_omega,
                  const double* omega_h, double eta, double* gre_h, double* gim_h) {
  double *a, *b, *om, *gr, *gi;
  CA(dalloc(c, &a, (size_t)m)); CA(dalloc(c, &b, (size_t)m)); CA(dalloc(c, &om, (size_t)n_omega));
  CA(dalloc(c, &gr, (size_t)n_omega)); CA(dalloc(c, &gi, (size_t)n_omega));
  struct G8 { bse_ctx* c; std::vector<void*> v; ~G8() { for (void* x : v) dfree(c, x); } } g8{c, {a, b, om, gr, gi}};
  CK(cudaMemcpyAsync(a, alpha_h, sizeof(double) * m, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(b, beta_h, sizeof(double) * m, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(om, omega_h, sizeof(double) * n_omega, cudaMemcpyHostToDevice, c->st));
  CK(continued_fraction(m, a, b, norm2, n_omega, om, eta, gr, gi, c->st));
  CK(cudaMemcpyAsync(gre_h, gr, sizeof(double) * n_omega, cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(gim_h, gi, sizeof(double) * n_omega, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  return BSE_OK;
}

// ---------------------------------------------------------------------------------
// Wannier localisation (Section 2, Eqs. wannier and spread): JADE on the six matrices
// A^(n) = <psi|M^(n)|psi>, then the context's orbitals become psi~ = U^T psi and the
// occupied energies the matrix U^T diag(eps) U
// ---------------------------------------------------------------------------------
// recompute everything derived from psi64: psi on the grid, the FP32 copies and the BF16
// splits of the mixed path
int refresh_orbitals(bse_ctx* c) {
  const long ng = (c->n_occ + 1) / 2, npsi = (long)c->n_occ * c->n_pw;
  CK((sphere_unpack<double, double>(c->psi64, c->n_occ, c->n_pw, c->n_half, c->gpos, c->gneg, (double2*)c->upsi64,
                                    c->n3, true, false, c->st)));
  CK(fft3d<double>((double2*)c->upsi64, ng, c->N, +1, c->tw64, c->st));
  if (c->prec == BSE_PREC_MIXED) {
    CK((convert<double, float>(ng * 2 * c->n3, c->upsi64, c->upsi32, c->st)));
    CK((convert<double, float>(npsi, c->psi64, c->psi32, c->st)));
    if (c->tc_ok) {
      CK(bf16_split64(c->psi64, c->n_occ, c->n_pw, c->n_pw, c->psi_s.hi, c->psi_s.lo, c->psi_s.ld, false, c->st));
      CK(bf16_split64(c->psi64, c->n_occ, c->n_pw, c->n_pw, c->psiT_s.hi, c->psiT_s.lo, c->psiT_s.ld, true, c->st));
    }
  }
  return BSE_OK;
}

int localize_impl(bse_ctx* c, int max_sweeps, double tol, double* U_out) {
  const int n = c->n_occ;
  const long n3 = c->n3;
  constexpr int K = 6;
  std::vector<void*> mine;
  auto al = [&](auto** p, size_t m) {
    int r = dalloc(c, p, m);
    if (r == BSE_OK) mine.push_back(*p);
    return r;
  };
  struct Guard {
    bse_ctx* c; std::vector<void*>* m;
    ~Guard() { for (void* p : *m) dfree(c, p); }
  } guard{c, &mine};
  double *u, *W, *A, *U, *Bd, *tmp;
  double2* cs;
  int2* pairs_d;
  unsigned* smax;
  CA(al(&u, (size_t)n * n3)); CA(al(&W, (size_t)n * n3)); CA(al(&A, (size_t)K * n * n));
  CA(al(&U, (size_t)n * n)); CA(al(&Bd, (size_t)K * n)); CA(al(&tmp, (size_t)n * c->n_pw));
  // A^(n) = N^-3 u M u^T and the diagonals of B^(n) (u = Omega^{1/2} psi on the grid; the
  // products are band-limited, so the grid sums are exact)
  CK(pair_grid_to_rows<double>(n, c->upsi64, n3, u, c->st));
  const double w = 1.0 / (double)n3;
  for (int op = 0; op < K; ++op) {
    CK(jade_weight(n, n3, c->N, op, u, W, false, c->st));
    CK((gemm<double, double>(false, true, n, n, (int)n3, w, u, n3, W, n3, 0.0, A + (size_t)op * n * n, n, 0, c->st)));
    CK(jade_weight(n, n3, c->N, op, u, W, true, c->st));
    CK(row_dots(n, n3, u, W, Bd + (size_t)op * n, c->st));
  }
  auto spread_now = [&](double& out) -> int {
    std::vector<double> hA((size_t)K * n * n), hB((size_t)K * n);
    CK(cudaMemcpyAsync(hA.data(), A, sizeof(double) * hA.size(), cudaMemcpyDeviceToHost, c->st));
    CK(cudaMemcpyAsync(hB.data(), Bd, sizeof(double) * hB.size(), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    double sg = 0;
    for (int op = 0; op < K; ++op)
      for (int v = 0; v < n; ++v) {
        const double d = hA[(size_t)op * n * n + (size_t)v * n + v];
        sg += w * hB[(size_t)op * n + v] - d * d;
      }
    out = sg;
    return BSE_OK;
  };
  CA(spread_now(c->spread0));
  // sweeps: first on A^(1) alone (its eigenvectors start U, as in the paper), then on all six
  std::vector<int2> sched;
  int rounds = 0, per = 0;
  jade_schedule(n, sched, rounds, per);
  CA(al(&pairs_d, sched.size())); CA(al(&cs, (size_t)per)); CA(al(&smax, 1));
  CK(cudaMemcpyAsync(pairs_d, sched.data(), sizeof(int2) * sched.size(), cudaMemcpyHostToDevice, c->st));
  CK(set_identity(n, U, c->st));
  for (int stage = 0; stage < 2; ++stage) {
    const int k_use = stage == 0 ? 1 : K;
    for (int sw = 0; sw < max_sweeps; ++sw) {
      CK(cudaMemsetAsync(smax, 0, sizeof(unsigned), c->st));
      for (int r = 0; r < rounds; ++r)
        CK(jade_round(k_use, K, n, A, U, pairs_d + (size_t)r * per, per, cs, smax, c->st));
      unsigned hs = 0;
      CK(cudaMemcpyAsync(&hs, smax, sizeof(unsigned), cudaMemcpyDeviceToHost, c->st));
      CK(cudaStreamSynchronize(c->st));
      float f;
      std::memcpy(&f, &hs, sizeof(f));
      if (!std::isfinite(f)) return fail(c, BSE_ERR_NUMERIC, "non-finite rotation in the localisation");
      if ((double)f <= tol) break;
    }
  }
  CA(spread_now(c->spread1));
  // psi~ = U^T psi; E = U^T diag(eps) U (diagonal -> eps, the rest -> the operator term)
  CK((gemm<double, double>(true, false, n, c->n_pw, n, 1.0, U, n, c->psi64, c->n_pw, 0.0, tmp, c->n_pw, 1, c->st)));
  CK(cudaMemcpyAsync(c->psi64, tmp, sizeof(double) * n * c->n_pw, cudaMemcpyDeviceToDevice, c->st));
  CA(refresh_orbitals(c));
  double *Ev, *E;
  CA(al(&Ev, (size_t)n)); CA(al(&E, (size_t)n * n));
  CK(cudaMemcpyAsync(Ev, c->eps_h.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(W, U, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, c->st));
  CK(scale_rows<double>(n, n, W, Ev, c->st));                                   // diag(eps) U
  CK((gemm<double, double>(true, false, n, n, n, 1.0, U, n, W, n, 0.0, E, n, 1, c->st)));
  std::vector<double> hE((size_t)n * n), hU((size_t)n * n);
  CK(cudaMemcpyAsync(hE.data(), E, sizeof(double) * hE.size(), cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(hU.data(), U, sizeof(double) * hU.size(), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (!all_finite(hE.data(), (long)n * n) || !all_finite(hU.data(), (long)n * n))
    return fail(c, BSE_ERR_NUMERIC, "non-finite localising rotation");
  std::vector<double> ediag(n), esh(n);
  for (int v = 0; v < n; ++v) { ediag[v] = hE[(size_t)v * n + v]; hE[(size_t)v * n + v] = 0.0; }
  c->eps_h = ediag;
  for (int v = 0; v < n; ++v) esh[v] = c->scissor - ediag[v];
  std::vector<float> eshf(esh.begin(), esh.end()), ef(hE.begin(), hE.end());
  CK(cudaMemcpyAsync(c->eps, ediag.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->esh64, esh.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->esh32, eshf.data(), sizeof(float) * n, cudaMemcpyHostToDevice, c->st));
  if (!c->eoff64) CA(dalloc(c, &c->eoff64, (size_t)n * n));
  if (!c->eoff32) CA(dalloc(c, &c->eoff32, (size_t)n * n));
  CK(cudaMemcpyAsync(c->eoff64, hE.data(), sizeof(double) * n * n, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->eoff32, ef.data(), sizeof(float) * n * n, cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  c->has_emat = true;
  if (U_out) std::memcpy(U_out, hU.data(), sizeof(double) * n * n);
  return BSE_OK;
}

}  // namespace

// =================================================================================
// C ABI
// =================================================================================
extern "C" {

const char* bse_version(void) {
  return "bse-gb300 0.1 (sm_103a; FP64 plain and FP32/FP64 mixed paths)";
}

const char* bse_last_error(const bse_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void bse_destroy(bse_ctx* ctx) {
  if (!ctx) return;
  for (void* p : ctx->allocs) dfree_raw(ctx, p);
  ctx->allocs.clear();
  cudaStreamSynchronize(ctx->st);
  delete ctx;
}

int bse_create(const bse_system* s, int precision, bse_alloc_fn alloc_fn, bse_free_fn free_fn, void* user,
               void* stream, bse_ctx** out) {
  if (!out) return BSE_ERR_INVALID_ARG;
  *out = nullptr;
  if (!s) return BSE_ERR_INVALID_ARG;
  if (precision != BSE_PREC_FP64 && precision != BSE_PREC_MIXED) return BSE_ERR_INVALID_ARG;
  if ((alloc_fn == nullptr) != (free_fn == nullptr)) return BSE_ERR_INVALID_ARG;
  bse_ctx* c = new bse_ctx();
  auto bail = [&](int code) { if (code != BSE_OK) { *out = c; } return code; };
  c->st = (cudaStream_t)stream;
  c->ua = alloc_fn;
  c->uf = free_fn;
  c->uu = user;
  c->prec = precision;
  if (!fft_supported(s->n_grid)) return bail(fail(c, BSE_ERR_INVALID_ARG, "n_grid must be one of 16, 32, 48, 64, 72, 96"));
  if (!(s->L > 0) || s->n_half < 1 || s->n_occ < 1 || s->n_pdep < 0 || !s->miller || !s->psi ||
      (!s->eps && s->n_qp == 0) || !s->v_loc || (s->n_pdep > 0 && (!s->pdep || !s->lambda)) ||
      (s->spin != 0 && s->spin != 1))
    return bail(fail(c, BSE_ERR_INVALID_ARG, "invalid system sizes or null pointers"));
  if (s->n_qp != 0 && (s->n_qp <= s->n_occ || !s->qp_psi || !s->qp_eps_ks || !s->qp_eps))
    return bail(fail(c, BSE_ERR_INVALID_ARG, "n_qp must be 0 or > n_occ, with qp_psi, qp_eps_ks and qp_eps"));
  if (s->overlap_thr <= 0 && s->keep_pairs < 1)
    return bail(fail(c, BSE_ERR_INVALID_ARG, "need overlap_thr > 0 or keep_pairs >= 1"));
  c->N = s->n_grid; c->n3 = (long)c->N * c->N * c->N; c->L = s->L; c->omega = s->L * s->L * s->L;
  c->n_half = s->n_half; c->n_pw = 2 * s->n_half; c->n_occ = s->n_occ; c->n_pdep = s->n_pdep;
  c->spin = s->spin; c->scissor = s->scissor; c->thr_in = s->overlap_thr; c->keep_pairs = s->keep_pairs;
  if (s->n_up < 0 || s->n_up > s->n_occ) return bail(fail(c, BSE_ERR_INVALID_ARG, "n_up must be in [0, n_occ]"));
  c->n_up = s->n_up;
  if (c->n_occ >= c->n_pw - 1) return bail(fail(c, BSE_ERR_INVALID_ARG, "n_occ must be smaller than the sphere dimension"));
  const int rmax = (c->N - 1) / 4;
  std::vector<int> gpos(c->n_half), gneg(c->n_half);
  for (int k = 0; k < c->n_half; ++k) {
    const int* m = &s->miller[3 * k];
    for (int a = 0; a < 3; ++a)
      if (m[a] > rmax || m[a] < -rmax)
        return bail(fail(c, BSE_ERR_INVALID_ARG, "miller index beyond (N-1)/4: products would alias"));
    if (k == 0 && (m[0] | m[1] | m[2])) return bail(fail(c, BSE_ERR_INVALID_ARG, "miller[0] must be (0,0,0)"));
    if (k > 0 && !(m[0] | m[1] | m[2])) return bail(fail(c, BSE_ERR_INVALID_ARG, "G = 0 appears twice"));
    auto idx = [&](int x, int y, int z) {
      x = (x % c->N + c->N) % c->N; y = (y % c->N + c->N) % c->N; z = (z % c->N + c->N) % c->N;
      return x + c->N * (y + c->N * z);
    };
    gpos[k] = idx(m[0], m[1], m[2]);
    gneg[k] = idx(-m[0], -m[1], -m[2]);
  }
  const long npsi = (long)c->n_occ * c->n_pw;
  c->n_qc = s->n_qp ? s->n_qp - s->n_occ : 0;
  if (!all_finite(s->psi, npsi) || (s->n_qp == 0 && (!all_finite(s->eps, c->n_occ) || !std::isfinite(s->scissor))) ||
      !all_finite(s->v_loc, c->n3) ||
      (c->n_pdep > 0 && (!all_finite(s->pdep, (long)c->n_pdep * c->n_pw) || !all_finite(s->lambda, c->n_pdep))) ||
      (c->n_qc > 0 && (!all_finite(s->qp_psi, (long)c->n_qc * c->n_pw) || !all_finite(s->qp_eps_ks, s->n_qp) ||
                       !all_finite(s->qp_eps, s->n_qp))))
    return bail(fail(c, BSE_ERR_NUMERIC, "non-finite input"));
  for (int q = 0; q < c->n_qc; ++q)
    if (s->qp_psi[(long)q * c->n_pw + 1] != 0.0) return bail(fail(c, BSE_ERR_INVALID_ARG, "qp_psi pad entry (index 1) must be 0"));
  // D of Eq. (d) with the QP Hamiltonian of Eq. (ham): occupied energies eps^QP_v, the uniform
  // shift Delta (the scissor, or the average of the QP corrections over N_mid..N_QP) and, with
  // explicit QP data, the corrections delta_c of the conduction states n_occ+1..N_QP
  std::vector<double> eps_use(c->n_occ), qdelta_h(std::max(1, c->n_qc), 0.0);
  if (c->n_qc > 0) {
    const int nqp = s->n_qp, n_mid = (s->n_occ + s->n_qp) / 2;
    double sum = 0;
    for (int n = n_mid - 1; n < nqp; ++n) sum += s->qp_eps[n] - s->qp_eps_ks[n];
    c->scissor = sum / (double)(nqp - n_mid + 1);
    for (int v = 0; v < c->n_occ; ++v) eps_use[v] = s->qp_eps[v];
    for (int q = 0; q < c->n_qc; ++q) qdelta_h[q] = s->qp_eps[c->n_occ + q] - s->qp_eps_ks[c->n_occ + q] - c->scissor;
  } else {
    for (int v = 0; v < c->n_occ; ++v) eps_use[v] = s->eps[v];
  }
  for (int v = 0; v < c->n_occ; ++v)
    if (s->psi[(long)v * c->n_pw + 1] != 0.0) return bail(fail(c, BSE_ERR_INVALID_ARG, "psi pad entry (index 1) must be 0"));
  for (int a = 0; a < c->n_pdep; ++a) {
    if (s->pdep[(long)a * c->n_pw] != 0.0 || s->pdep[(long)a * c->n_pw + 1] != 0.0)
      return bail(fail(c, BSE_ERR_INVALID_ARG, "pdep entries 0 and 1 must be 0"));
    if (!(s->lambda[a] < 1.0)) return bail(fail(c, BSE_ERR_INVALID_ARG, "lambda must be < 1"));
  }
  // host tables
  const double g = 2.0 * M_PI / c->L;
  c->g2p_h.assign(c->n_pw, 0.0);
  c->gcart_h.assign((size_t)3 * c->n_pw, 0.0);
  for (int k = 0; k < c->n_half; ++k) {
    const int* m = &s->miller[3 * k];
    const double g2 = g * g * (double)(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
    c->g2p_h[2 * k] = g2;
    c->g2p_h[2 * k + 1] = (k == 0) ? 0.0 : g2;
    for (int a = 0; a < 3; ++a) c->gcart_h[(size_t)a * c->n_pw + 2 * k] = c->gcart_h[(size_t)a * c->n_pw + 2 * k + 1] =
        (k == 0) ? 0.0 : g * (double)m[a];
  }
  c->eps_h = eps_use;
  double vs = 0;
  for (long r = 0; r < c->n3; ++r) vs += s->v_loc[r];
  c->v0 = vs / (double)c->n3;
  std::vector<double> fh(std::max(1, c->n_pdep), 0.0);
  for (int a = 0; a < c->n_pdep; ++a) fh[a] = s->lambda[a] / (1.0 - s->lambda[a]);
  // workspace budget: BSE_WORKSPACE_GB or 40% of free memory, at most 64 GB
  {
    size_t fr = 0, tot = 0;
    const cudaError_t em = cudaMemGetInfo(&fr, &tot);
    if (em != cudaSuccess) return bail(cuda_fail(c, em, "cudaMemGetInfo"));
    size_t bud = std::min<size_t>((size_t)64 << 30, (size_t)(0.4 * (double)fr));
    if (const char* e = getenv("BSE_WORKSPACE_GB")) bud = (size_t)(atof(e) * (double)(1ull << 30));
    if (const char* e = getenv("BSE_AUTOTUNE")) c->autotune = atoi(e) != 0;
    if (const char* e = getenv("BSE_TC_WAIT_LIMIT")) c->tc_wait_limit = atoll(e);
    // BSE_K1D_VARIANT=v fixes the K1d tile variant (no autotuning); ignored if it does not fit
    if (const char* e = getenv("BSE_K1D_VARIANT")) {
      const int v = atoi(e);
      const bool ok = (precision == BSE_PREC_FP64) ? k1d_fits<double>(s->n_occ, v) : k1d_fits<float>(s->n_occ, v);
      if (ok) c->k1d_force = v;
    }
    // BSE_K1D_SYM_VARIANT=v does the same for the kernel of tau stored once per pair
    if (const char* e = getenv("BSE_K1D_SYM_VARIANT")) {
      const int v = atoi(e);
      const bool ok = (precision == BSE_PREC_FP64) ? k1d_sym_fits<double>(s->n_occ, v) : k1d_sym_fits<float>(s->n_occ, v);
      if (ok) c->k1d_force_sym = v;
    }
    c->ws_budget = std::max<size_t>(bud, 1);
  }
  // device uploads
#define UPLOAD(dst, src, n)                                                                    \
  do {                                                                                         \
    int _r = dalloc(c, &(dst), (size_t)(n));                                                   \
    if (_r != BSE_OK) return bail(_r);                                                         \
    cudaError_t _e = cudaMemcpyAsync(dst, src, sizeof(*(dst)) * (size_t)(n), cudaMemcpyHostToDevice, c->st); \
    if (_e != cudaSuccess) return bail(cuda_fail(c, _e, "upload"));                            \
  } while (0)
  UPLOAD(c->gpos, gpos.data(), c->n_half);
  UPLOAD(c->gneg, gneg.data(), c->n_half);
  {
    SphereMapHost h;
    build_sphere_map(c->N, c->n_half, s->miller, h);
    if (sphere_scratch_per_grid(c->N, SphereMap{h.NS, h.NC, h.NX}) > (size_t)c->n3)
      return bail(fail(c, BSE_ERR_INVALID_ARG, "sphere too large for the pruned transforms"));
    int *fp, *fn, *zs, *jc, *cs, *cy, *cx, *xs, *xc;
    UPLOAD(fp, h.fpos.data(), h.fpos.size());
    UPLOAD(fn, h.fneg.data(), h.fneg.size());
    UPLOAD(zs, h.zs.data(), h.zs.size());
    UPLOAD(jc, h.jcol.data(), h.jcol.size());
    UPLOAD(cs, h.cstart.data(), h.cstart.size());
    UPLOAD(cy, h.cy.data(), h.cy.size());
    UPLOAD(cx, h.cxi.data(), h.cxi.size());
    UPLOAD(xs, h.xs.data(), h.xs.size());
    UPLOAD(xc, h.xcol.data(), h.xcol.size());
    c->sph = SphereMap{h.NS, h.NC, h.NX, fp, fn, zs, jc, cs, cy, cx, xs, xc};
  }
  UPLOAD(c->g2p, c->g2p_h.data(), c->n_pw);
  UPLOAD(c->eps, eps_use.data(), c->n_occ);
  if (c->n_qc > 0) {
    UPLOAD(c->qpsi64, s->qp_psi, (long)c->n_qc * c->n_pw);
    UPLOAD(c->qdelta, qdelta_h.data(), c->n_qc);
  }
  {
    std::vector<double> g2h(c->n_pw), esh(c->n_occ);
    for (int j = 0; j < c->n_pw; ++j) g2h[j] = 0.5 * c->g2p_h[j];
    for (int v = 0; v < c->n_occ; ++v) esh[v] = c->scissor - eps_use[v];
    std::vector<float> g2hf(g2h.begin(), g2h.end()), eshf(esh.begin(), esh.end());
    UPLOAD(c->g2h64, g2h.data(), g2h.size());
    UPLOAD(c->esh64, esh.data(), esh.size());
    UPLOAD(c->g2h32, g2hf.data(), g2hf.size());
    UPLOAD(c->esh32, eshf.data(), eshf.size());
  }
  UPLOAD(c->f, fh.data(), fh.size());
  UPLOAD(c->psi64, s->psi, npsi);
  c->occw_h.assign((size_t)2 * c->n_pw, 0.0);
  for (int v = 0; v < c->n_occ; ++v)
    for (int j = 0; j < c->n_pw; ++j)
      c->occw_h[(size_t)c->chan(v) * c->n_pw + j] += s->psi[(long)v * c->n_pw + j] * s->psi[(long)v * c->n_pw + j];
  UPLOAD(c->vloc64, s->v_loc, c->n3);
  if (c->n_pdep > 0) UPLOAD(c->pdep64, s->pdep, (long)c->n_pdep * c->n_pw);
  std::vector<double2> tw;
  twiddle_table(c->N, tw);
  UPLOAD(c->tw64, tw.data(), tw.size());
  std::vector<float2> twf(tw.size());
  for (size_t i = 0; i < tw.size(); ++i) { twf[i].x = (float)tw[i].x; twf[i].y = (float)tw[i].y; }
  UPLOAD(c->tw32, twf.data(), twf.size());
  {
    int r0 = dalloc(c, &c->d_bad, 1);
    if (r0 != BSE_OK) return bail(r0);
  }
  // psi_v(r) (times Omega^{1/2}) in FP64 on the grid, pair layout
  {
    const long ng = (c->n_occ + 1) / 2;
    double2* up;
    int r = dalloc(c, &up, (size_t)ng * c->n3);
    if (r != BSE_OK) return bail(r);
    cudaError_t e = sphere_unpack<double, double>(c->psi64, c->n_occ, c->n_pw, c->n_half, c->gpos,
                                                  c->gneg, up, c->n3, true, false, c->st);
    if (e == cudaSuccess) e = fft3d<double>(up, ng, c->N, +1, c->tw64, c->st);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "psi to real space"));
    c->upsi64 = (double*)up;
    if (c->prec == BSE_PREC_MIXED) {
      const long nr = ng * 2 * c->n3;
      if ((r = dalloc(c, &c->upsi32, (size_t)nr)) != BSE_OK) return bail(r);
      if ((r = dalloc(c, &c->psi32, (size_t)npsi)) != BSE_OK) return bail(r);
      if ((r = dalloc(c, &c->vloc32, (size_t)c->n3)) != BSE_OK) return bail(r);
      e = convert<double, float>(nr, c->upsi64, c->upsi32, c->st);
      if (e == cudaSuccess) e = convert<double, float>(npsi, c->psi64, c->psi32, c->st);
      if (e == cudaSuccess) e = convert<double, float>(c->n3, c->vloc64, c->vloc32, c->st);
      if (e == cudaSuccess && c->n_pdep > 0) {
        if ((r = dalloc(c, &c->pdep32, (size_t)c->n_pdep * c->n_pw)) != BSE_OK) return bail(r);
        e = convert<double, float>((long)c->n_pdep * c->n_pw, c->pdep64, c->pdep32, c->st);
      }
      if (e == cudaSuccess && c->n_qc > 0) {
        if ((r = dalloc(c, &c->qpsi32, (size_t)c->n_qc * c->n_pw)) != BSE_OK) return bail(r);
        e = convert<double, float>((long)c->n_qc * c->n_pw, c->qpsi64, c->qpsi32, c->st);
      }
      if (e != cudaSuccess) return bail(cuda_fail(c, e, "FP32 copies"));
      // BF16x3 tensor-core operands: Psi, Psi^T, Phi, Phi^T split once
      if ((r = dalloc(c, &c->d_err, 1)) != BSE_OK) return bail(r);
      if ((e = cudaMemsetAsync(c->d_err, 0, sizeof(int), c->st)) != cudaSuccess) return bail(cuda_fail(c, e, "err flag"));
      if (tc_map_bytes() == sizeof(TMap) && getenv("BSE_NO_TENSOR_CORES") == nullptr) {
        int rr = make_split64(c, c->psi_s, c->psi64, c->n_occ, c->n_pw, false);
        if (rr == BSE_OK) rr = make_split64(c, c->psiT_s, c->psi64, c->n_occ, c->n_pw, true);
        if (rr == BSE_OK && c->n_pdep > 0) rr = make_split64(c, c->pdep_s, c->pdep64, c->n_pdep, c->n_pw, false);
        if (rr == BSE_OK && c->n_pdep > 0) rr = make_split64(c, c->pdepT_s, c->pdep64, c->n_pdep, c->n_pw, true);
        if (rr == BSE_OK && c->n_qc > 0) rr = make_split64(c, c->qpsi_s, c->qpsi64, c->n_qc, c->n_pw, false);
        if (rr == BSE_OK && c->n_qc > 0) rr = make_split64(c, c->qpsiT_s, c->qpsi64, c->n_qc, c->n_pw, true);
        if (rr != BSE_OK) return bail(rr);
        c->tc_ok = true;
      }
    }
  }
  cudaError_t e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "bse_create"));
  *out = c;
  return BSE_OK;
}

static int check_device_flag(bse_ctx* c) {
  if (!c->d_err) return BSE_OK;
  int h = 0;
  if (cudaMemcpy(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return BSE_OK;
  if (h) {
    cudaMemset(c->d_err, 0, sizeof(int));
    return fail(c, BSE_ERR_TIMEOUT, "a bounded device wait gave up (tensor-core pipeline)");
  }
  return BSE_OK;
}

int bse_build_tau(bse_ctx* c, int64_t* n_pairs_out, double* thr_out) {
  if (!c) return BSE_ERR_INVALID_ARG;
  int r = (c->prec == BSE_PREC_FP64) ? build_tau_impl<double>(c) : build_tau_impl<float>(c);
  cudaStreamSynchronize(c->st);
  c->prof.resolve();
  if (r != BSE_OK) return r;
  if ((r = check_device_flag(c)) != BSE_OK) return r;
  if (n_pairs_out) *n_pairs_out = c->n_pairs;
  if (thr_out) *thr_out = c->thr;
  return BSE_OK;
}

int bse_get_pairs(const bse_ctx* c, int32_t* v_out, int32_t* w_out) {
  if (!c || !v_out || !w_out) return BSE_ERR_INVALID_ARG;
  if (!c->tau_ready) return BSE_ERR_STATE;
  std::memcpy(v_out, c->pv_h.data(), sizeof(int32_t) * c->pv_h.size());
  std::memcpy(w_out, c->pw_h.data(), sizeof(int32_t) * c->pw_h.size());
  return BSE_OK;
}

int bse_get_overlaps(const bse_ctx* c, double* o_out) {
  if (!c || !o_out) return BSE_ERR_INVALID_ARG;
  if (c->O_h.empty()) return BSE_ERR_STATE;
  std::memcpy(o_out, c->O_h.data(), sizeof(double) * c->O_h.size());
  return BSE_OK;
}

int bse_apply_liouville(bse_ctx* c, int n_vec, const void* a_in, void* a_out) {
  if (!c) return BSE_ERR_INVALID_ARG;
  if (n_vec < 0 || (n_vec > 0 && (!a_in || !a_out))) return fail(c, BSE_ERR_INVALID_ARG, "bad apply arguments");
  if (a_in == a_out && n_vec > 0) return fail(c, BSE_ERR_INVALID_ARG, "a_out must not alias a_in");
  if (!c->tau_ready) return fail(c, BSE_ERR_STATE, "bse_build_tau must run before bse_apply_liouville");
  int r = (c->prec == BSE_PREC_FP64)
              ? apply_impl<double>(c, n_vec, (const double*)a_in, (double*)a_out)
              : apply_impl<float>(c, n_vec, (const float*)a_in, (float*)a_out);
  if (r != BSE_OK) return r;
  cudaError_t e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return cuda_fail(c, e, "bse_apply_liouville");
  c->prof.resolve();
  return check_device_flag(c);
}

int bse_davidson(bse_ctx* c, const bse_davidson_opts* o, double* omega_out, void* vec_out,
                 bse_davidson_stats* stats) {
  if (!c) return BSE_ERR_INVALID_ARG;
  if (!o || !omega_out) return fail(c, BSE_ERR_INVALID_ARG, "null options or omega_out");
  if (!c->tau_ready) return fail(c, BSE_ERR_STATE, "bse_build_tau must run before bse_davidson");
  int r = (c->prec == BSE_PREC_FP64)
              ? davidson_impl<double>(c, o, omega_out, (double*)vec_out, stats)
              : davidson_impl<float>(c, o, omega_out, (float*)vec_out, stats);
  cudaStreamSynchronize(c->st);
  c->prof.resolve();
  if (r == BSE_OK || r == BSE_ERR_NOT_CONVERGED) {
    const int f = check_device_flag(c);
    if (f != BSE_OK) return f;
  }
  return r;
}

int bse_localize(bse_ctx* c, int max_sweeps, double tol, double* U_out, double* spread_out) {
  if (!c) return BSE_ERR_INVALID_ARG;
  if (max_sweeps < 1 || !(tol > 0)) return fail(c, BSE_ERR_INVALID_ARG, "bse_localize: max_sweeps >= 1, tol > 0");
  if (c->tau_ready) return fail(c, BSE_ERR_STATE, "bse_localize must run before bse_build_tau");
  if (c->n_up > 0) return fail(c, BSE_ERR_INVALID_ARG, "bse_localize: closed-shell systems only");
  int r = localize_impl(c, max_sweeps, tol, U_out);
  cudaStreamSynchronize(c->st);
  if (r != BSE_OK) return r;
  if (spread_out) { spread_out[0] = c->spread0; spread_out[1] = c->spread1; }
  return BSE_OK;
}

int bse_lanczos(bse_ctx* c, int n_pol, const int* dirs, int n_steps, double* alpha_out, double* beta_out,
                double* norm2_out) {
  if (!c) return BSE_ERR_INVALID_ARG;
  if (n_pol < 1 || n_pol > 3 || !dirs || n_steps < 1 || !alpha_out || !beta_out || !norm2_out)
    return fail(c, BSE_ERR_INVALID_ARG, "bse_lanczos: need 1 <= n_pol <= 3, dirs, n_steps >= 1 and outputs");
  for (int p = 0; p < n_pol; ++p)
    if (dirs[p] < 0 || dirs[p] > 2) return fail(c, BSE_ERR_INVALID_ARG, "bse_lanczos: directions are 0, 1, 2");
  if (!c->tau_ready) return fail(c, BSE_ERR_STATE, "bse_build_tau must run before bse_lanczos");
  int r = (c->prec == BSE_PREC_FP64)
              ? lanczos_impl<double>(c, n_pol, dirs, n_steps, alpha_out, beta_out, norm2_out)
              : lanczos_impl<float>(c, n_pol, dirs, n_steps, alpha_out, beta_out, norm2_out);
  cudaStreamSynchronize(c->st);
  c->prof.resolve();
  if (r != BSE_OK) return r;
  return check_device_flag(c);
}

int bse_lanczos_spectrum(bse_ctx* c, int n_steps, const double* alpha, const double* beta, double norm2,
                         int n_omega, const double* omega, double eta, double* g_re, double* g_im) {
  if (!c) return BSE_ERR_INVALID_ARG;
  if (n_steps < 1 || !alpha || !beta || n_omega < 0 || (n_omega > 0 && (!omega || !g_re || !g_im)) || !(eta > 0))
    return fail(c, BSE_ERR_INVALID_ARG, "bse_lanczos_spectrum: bad arguments (eta must be > 0)");
  if (n_omega == 0) return BSE_OK;
  return spectrum_impl(c, n_steps, alpha, beta, norm2, n_omega, omega, eta, g_re, g_im);
}

int bse_solve_batch(bse_ctx* const* ctxs, int n, const bse_davidson_opts* o, double* omega_out,
                    bse_davidson_stats* stats, int* status_out) {
  if (!ctxs || n < 1 || !o || !omega_out) return BSE_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i)
    if (!ctxs[i]) return BSE_ERR_INVALID_ARG;
  int dev = 0;
  cudaGetDevice(&dev);
  std::vector<int> rc(n, BSE_OK);
  // A pool of worker threads takes the systems in order from a shared counter (at most
  // BSE_BATCH_WORKERS at a time, default 16), each driving its context's stream, so the
  // number of systems holding workspaces at once stays bounded. A system whose solve ran out
  // of device memory is solved again after the pool has finished, alone.
  int workers = 16;
  if (const char* e = getenv("BSE_BATCH_WORKERS")) workers = std::max(1, atoi(e));
  workers = std::min(workers, n);
  std::atomic<int> next{0};
  auto solve_one = [&](int i) {
    bse_ctx* c = ctxs[i];
    int r = BSE_OK;
    if (!c->tau_ready) r = bse_build_tau(c, nullptr, nullptr);
    if (r == BSE_OK) r = bse_davidson(c, o, omega_out + (size_t)i * o->n_eig, nullptr, stats ? stats + i : nullptr);
    rc[i] = r;
  };
  std::vector<std::thread> th;
  th.reserve(workers);
  for (int k = 0; k < workers; ++k) {
    th.emplace_back([&] {
      cudaSetDevice(dev);
      for (int i = next++; i < n; i = next++) solve_one(i);
    });
  }
  for (auto& t : th) t.join();
  for (int i = 0; i < n; ++i)
    if (rc[i] == BSE_ERR_OOM) solve_one(i);
  int first = BSE_OK;
  for (int i = 0; i < n; ++i) {
    if (status_out) status_out[i] = rc[i];
    if (first == BSE_OK && rc[i] != BSE_OK) first = rc[i];
  }
  return first;
}

int bse_profile(bse_ctx* c, int mode) {
  if (!c) return BSE_ERR_INVALID_ARG;
  cudaStreamSynchronize(c->st);
  c->prof.resolve();
  if (mode == 1) c->prof.on = true;
  else if (mode == 0) c->prof.on = false;
  else if (mode == -1) c->prof.acc.clear();
  else return fail(c, BSE_ERR_INVALID_ARG, "bse_profile mode must be 1, 0 or -1");
  return BSE_OK;
}

int bse_profile_read(bse_ctx* c, bse_prof_entry* out, int cap, int* n_out, int64_t* launches) {
  if (!c) {   // launch count only
    if (n_out) *n_out = 0;
    if (launches) *launches = (int64_t)launch_count();
    return launches ? BSE_OK : BSE_ERR_INVALID_ARG;
  }
  cudaStreamSynchronize(c->st);
  c->prof.resolve();
  if (out)
    for (int i = 0; i < cap && i < (int)c->prof.acc.size(); ++i) out[i] = c->prof.acc[i];
  if (n_out) *n_out = (int)c->prof.acc.size();
  if (launches) *launches = (int64_t)launch_count();
  return BSE_OK;
}

}  // extern "C"

// =================================================================================
// Learned preconditioner: samples, loss/gradient, training, loading
// =================================================================================
namespace {

void lp_free_samples(bse_ctx* c) {
  dfree(c, c->lp_r); dfree(c, c->lp_t); dfree(c, c->lp_theta); dfree(c, c->lp_rn2); dfree(c, c->lp_tn2);
  dfree(c, c->lp_u);
  c->lp_r = c->lp_t = c->lp_theta = c->lp_rn2 = c->lp_tn2 = c->lp_u = nullptr;
  c->lp_ns = 0;
}

int lp_alloc_samples(bse_ctx* c, long ns) {
  lp_free_samples(c);
  const long dim = (long)c->n_occ * c->n_pw;
  CA(dalloc(c, &c->lp_r, (size_t)ns * dim));
  CA(dalloc(c, &c->lp_t, (size_t)ns * dim));
  CA(dalloc(c, &c->lp_theta, (size_t)ns));
  CA(dalloc(c, &c->lp_rn2, (size_t)ns));
  CA(dalloc(c, &c->lp_tn2, (size_t)ns));
  c->lp_ns = ns;
  return BSE_OK;
}

int lp_finish_samples(bse_ctx* c) {
  const long dim = (long)c->n_occ * c->n_pw;
  CK(row_norms2<double>((int)c->lp_ns, dim, c->lp_r, c->lp_rn2, c->st));
  CK(row_norms2<double>((int)c->lp_ns, dim, c->lp_t, c->lp_tn2, c->st));
  return BSE_OK;
}

// one pass over the context's samples: loss (mean over samples, times `weight`) into d_loss
// and its gradient added into d_grad (double, mlpl::N)
int lp_step(bse_ctx* c, const float* d_params, int bf, double* d_grad, double* d_loss) {
  using namespace mlpl;
  const long ns = c->lp_ns, dim = (long)c->n_occ * c->n_pw, rows = ns * dim;
  std::vector<void*> tmp;
  auto al = [&](auto** p, size_t n) { int r = dalloc(c, p, n); if (r == BSE_OK) tmp.push_back(*p); return r; };
  struct G2 { bse_ctx* c; std::vector<void*>* t; ~G2() { for (void* p : *t) dfree(c, p); } } guard{c, &tmp};
  float *X, *H1, *H2, *O, *DO, *DZ1, *DZ2, *ones;
  double *Gv, *Y, *dg, *cb, *ab, *bb;
  CA(al(&X, (size_t)rows * F)); CA(al(&H1, (size_t)rows * H)); CA(al(&H2, (size_t)rows * H));
  CA(al(&O, (size_t)rows)); CA(al(&DO, (size_t)rows)); CA(al(&DZ1, (size_t)rows * H));
  CA(al(&DZ2, (size_t)rows * H)); CA(al(&ones, (size_t)rows)); CA(al(&Gv, (size_t)rows));
  CA(al(&Y, (size_t)rows)); CA(al(&dg, (size_t)rows));
  CA(al(&cb, (size_t)ns * c->n_occ * c->n_occ));
  CA(al(&ab, (size_t)2 * ns)); CA(al(&bb, (size_t)ns));
  std::vector<float> h1(rows, 1.0f);
  CK(cudaMemcpyAsync(ones, h1.data(), sizeof(float) * rows, cudaMemcpyHostToDevice, c->st));
  CK(mlp_train_forward(d_params, rows, c->n_occ, c->n_pw, c->lp_r, c->lp_theta, c->lp_rn2, c->g2p,
                       c->eps, c->v0, c->scissor, bf, X, H1, H2, O, Gv, Y, c->st));
  CA(project<double>(c, ns * c->n_occ, Y, cb));        // Y <- P_c(g r)
  // per sample a = <y, t*> and b = |y|^2, interleaved as (a, b)
  CK(row_dots((int)ns, dim, Y, c->lp_t, bb, c->st));
  CK(cudaMemcpy2DAsync(ab, 2 * sizeof(double), bb, sizeof(double), sizeof(double), ns, cudaMemcpyDeviceToDevice, c->st));
  CK(row_norms2<double>((int)ns, dim, Y, bb, c->st));
  CK(cudaMemcpy2DAsync(ab + 1, 2 * sizeof(double), bb, sizeof(double), sizeof(double), ns, cudaMemcpyDeviceToDevice, c->st));
  CK(mlp_loss(rows, dim, Y, c->lp_t, c->lp_tn2, ab, c->lp_r, 1.0 / (double)ns, dg, d_loss, c->st));
  CK(mlp_train_backward(d_params, rows, H1, H2, O, Gv, dg, DO, DZ1, DZ2, c->st));
  // d_grad += the parameter gradients (the products accumulate into it, beta = 1)
  CK((gemm<float, double>(true, false, H, F, (int)rows, 1.0, DZ1, H, X, F, 1.0, d_grad + W1, F, 0, c->st)));
  CK((gemm<float, double>(true, false, 1, H, (int)rows, 1.0, ones, 1, DZ1, H, 1.0, d_grad + B1, H, 0, c->st)));
  CK((gemm<float, double>(true, false, H, H, (int)rows, 1.0, DZ2, H, H1, H, 1.0, d_grad + W2, H, 0, c->st)));
  CK((gemm<float, double>(true, false, 1, H, (int)rows, 1.0, ones, 1, DZ2, H, 1.0, d_grad + B2, H, 0, c->st)));
  CK((gemm<float, double>(true, false, 1, H, (int)rows, 1.0, DO, 1, H2, H, 1.0, d_grad + W3, H, 0, c->st)));
  CK((gemm<float, double>(true, false, 1, 1, (int)rows, 1.0, ones, 1, DO, 1, 1.0, d_grad + B3, 1, 0, c->st)));
  return BSE_OK;
}

}  // namespace

extern "C" {

int bse_precond_set_samples(bse_ctx* c, int n, const double* r, const double* t, const double* theta) {
  if (!c) return BSE_ERR_INVALID_ARG;
  if (n < 1 || !r || !t || !theta) return fail(c, BSE_ERR_INVALID_ARG, "bse_precond_set_samples: bad arguments");
  const long dim = (long)c->n_occ * c->n_pw;
  if (!all_finite(r, n * dim) || !all_finite(t, n * dim) || !all_finite(theta, n))
    return fail(c, BSE_ERR_NUMERIC, "non-finite training sample");
  CA(lp_alloc_samples(c, n));
  CK(cudaMemcpyAsync(c->lp_r, r, sizeof(double) * n * dim, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->lp_t, t, sizeof(double) * n * dim, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->lp_theta, theta, sizeof(double) * n, cudaMemcpyHostToDevice, c->st));
  CA(lp_finish_samples(c));
  CK(cudaStreamSynchronize(c->st));
  return BSE_OK;
}

int bse_precond_collect(bse_ctx* c, const bse_davidson_opts* o, int ref_eig, int max_samples, int* n_out) {
  if (!c) return BSE_ERR_INVALID_ARG;
  if (!o || ref_eig < 1 || ref_eig > 32 || max_samples < 1)
    return fail(c, BSE_ERR_INVALID_ARG, "bse_precond_collect: need options, 1 <= ref_eig <= 32, max_samples >= 1");
  if (c->prec != BSE_PREC_FP64) return fail(c, BSE_ERR_STATE, "bse_precond_collect needs an FP64 context");
  if (!c->tau_ready) return fail(c, BSE_ERR_STATE, "bse_build_tau must run first");
  const long dim = (long)c->n_occ * c->n_pw;
  // reference eigenpairs of the plain solver
  double *Xr, *lam;
  CA(dalloc(c, &Xr, (size_t)ref_eig * dim));
  CA(dalloc(c, &lam, (size_t)ref_eig));
  struct G3 { bse_ctx* c; void* a; void* b; ~G3() { dfree(c, a); dfree(c, b); } } g3{c, Xr, lam};
  bse_davidson_opts ro{ref_eig, std::max(8, ref_eig), std::min(160, 4 * ref_eig + 32), 1000, 1e-8, 0};
  std::vector<double> lh(ref_eig);
  int r = davidson_impl<double>(c, &ro, lh.data(), Xr, nullptr);
  if (r != BSE_OK) return r;
  CK(cudaMemcpyAsync(lam, lh.data(), sizeof(double) * ref_eig, cudaMemcpyHostToDevice, c->st));
  // sampling run with the diagonal preconditioner: residuals, Ritz vectors and values
  double *U, *R;
  CA(dalloc(c, &U, (size_t)max_samples * dim));
  CA(dalloc(c, &R, (size_t)max_samples * dim));
  struct G4 { bse_ctx* c; void* a; void* b; ~G4() { dfree(c, a); dfree(c, b); } } g4{c, U, R};
  std::vector<double> thetas;
  SampleHook<double> hook = [&](int, const double* X, const double* Rr, const std::vector<double>& th,
                                const std::vector<int>& todo) -> int {
    for (int i : todo) {
      if ((long)thetas.size() >= max_samples) break;
      const long s = (long)thetas.size();
      CK(cudaMemcpyAsync(U + s * dim, X + (long)i * dim, sizeof(double) * dim, cudaMemcpyDeviceToDevice, c->st));
      CK(cudaMemcpyAsync(R + s * dim, Rr + (long)i * dim, sizeof(double) * dim, cudaMemcpyDeviceToDevice, c->st));
      thetas.push_back(th[i]);
    }
    return BSE_OK;
  };
  bse_davidson_opts so = *o;
  so.precond = 0;
  std::vector<double> om(so.n_eig);
  r = davidson_impl<double>(c, &so, om.data(), nullptr, nullptr, &hook);
  if (r != BSE_OK && r != BSE_ERR_NOT_CONVERGED) return r;
  const int ns = (int)thetas.size();
  if (ns == 0) return fail(c, BSE_ERR_STATE, "no samples: the solver converged before any correction");
  // Exact Jacobi-Davidson targets t* = y/(u.y) - u with y = (L - theta)^{-1} u. The part of
  // y in the span of the reference eigenvectors is the exact sum
  // sum_j x_j (x_j.u)/(lambda_j - theta); the rest z solves (L - theta) z = u - X X^T u on
  // the complement of that span, where L - theta is positive definite (theta lies below the
  // eigenvalues not in the reference set), by conjugate gradients with deflation, every
  // sample a column of one block (one operator application per CG iteration).
  CA(lp_alloc_samples(c, ns));
  double *Cm, *uy, *th_d, *Z, *Rc, *Pc, *Qc, *coef, *dots;
  CA(dalloc(c, &Cm, (size_t)ns * ref_eig));
  CA(dalloc(c, &uy, (size_t)ns));
  CA(dalloc(c, &th_d, (size_t)ns));
  CA(dalloc(c, &Z, (size_t)ns * dim)); CA(dalloc(c, &Rc, (size_t)ns * dim));
  CA(dalloc(c, &Pc, (size_t)ns * dim)); CA(dalloc(c, &Qc, (size_t)ns * dim));
  CA(dalloc(c, &coef, (size_t)ns)); CA(dalloc(c, &dots, (size_t)ns));
  struct G5 { bse_ctx* c; std::vector<void*> v; ~G5() { for (void* x : v) dfree(c, x); } } g5{c, {Cm, uy, th_d, Z, Rc, Pc, Qc, coef, dots}};
  CK(cudaMemcpyAsync(th_d, thetas.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, c->st));
  // low part: y_low = X diag(1/(lambda - theta)) X^T u (into lp_t)
  CK((gemm<double, double>(false, true, ns, ref_eig, (int)dim, 1.0, U, dim, Xr, dim, 0.0, Cm, ref_eig, 0, c->st)));
  // rhs of the complement: b = u - X (X^T u) (into Rc), before Cm is scaled
  CK(cudaMemcpyAsync(Rc, U, sizeof(double) * ns * dim, cudaMemcpyDeviceToDevice, c->st));
  CK((gemm<double, double>(false, false, ns, (int)dim, ref_eig, -1.0, Cm, ref_eig, Xr, dim, 1.0, Rc, dim, 1, c->st)));
  CK(shift_scale(ns, ref_eig, Cm, lam, th_d, c->st));
  CK((gemm<double, double>(false, false, ns, (int)dim, ref_eig, 1.0, Cm, ref_eig, Xr, dim, 0.0, c->lp_t, dim, 1, c->st)));
  // CG: z = 0, r = b, p = r
  CK(cudaMemsetAsync(Z, 0, sizeof(double) * ns * dim, c->st));
  CK(cudaMemcpyAsync(Pc, Rc, sizeof(double) * ns * dim, cudaMemcpyDeviceToDevice, c->st));
  std::vector<double> rr(ns), rr0(ns), pq(ns), hc(ns);
  CK(row_norms2<double>(ns, dim, Rc, dots, c->st));
  CK(cudaMemcpyAsync(rr.data(), dots, sizeof(double) * ns, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  rr0 = rr;
  std::vector<char> done(ns, 0);
  const double cg_tol = 1e-12;
  int cg_it = 0;
  for (; cg_it < 2000; ++cg_it) {
    bool all = true;
    for (int i = 0; i < ns; ++i) {
      if (!done[i] && rr[i] <= cg_tol * cg_tol * rr0[i]) done[i] = 1;
      all = all && done[i];
    }
    if (all) break;
    // q = (L - theta) p, deflated
    CA(apply_impl<double>(c, ns, Pc, Qc));
    CK(lanczos_axpy<double>(ns, dim, Qc, Pc, th_d, 1, nullptr, 0, c->st));
    CK((gemm<double, double>(false, true, ns, ref_eig, (int)dim, 1.0, Qc, dim, Xr, dim, 0.0, Cm, ref_eig, 0, c->st)));
    CK((gemm<double, double>(false, false, ns, (int)dim, ref_eig, -1.0, Cm, ref_eig, Xr, dim, 1.0, Qc, dim, 1, c->st)));
    CK(row_dots(ns, dim, Pc, Qc, dots, c->st));
    CK(cudaMemcpyAsync(pq.data(), dots, sizeof(double) * ns, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    // z += alpha p, r -= alpha q (alpha = 0 for converged columns)
    for (int i = 0; i < ns; ++i) hc[i] = (done[i] || !(pq[i] > 0)) ? 0.0 : -rr[i] / pq[i];
    CK(cudaMemcpyAsync(coef, hc.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, c->st));
    CK(lanczos_axpy<double>(ns, dim, Z, Pc, coef, 1, nullptr, 0, c->st));
    for (int i = 0; i < ns; ++i) hc[i] = -hc[i];
    CK(cudaMemcpyAsync(coef, hc.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, c->st));
    CK(lanczos_axpy<double>(ns, dim, Rc, Qc, coef, 1, nullptr, 0, c->st));
    CK(row_norms2<double>(ns, dim, Rc, dots, c->st));
    std::vector<double> rn(ns);
    CK(cudaMemcpyAsync(rn.data(), dots, sizeof(double) * ns, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    // p = r + beta p
    for (int i = 0; i < ns; ++i) hc[i] = (done[i] || !(rr[i] > 0)) ? 1.0 : rn[i] / rr[i];
    CK(cudaMemcpyAsync(coef, hc.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, c->st));
    CK(scale_rows<double>(ns, dim, Pc, coef, c->st));
    for (int i = 0; i < ns; ++i) hc[i] = done[i] ? 0.0 : -1.0;
    CK(cudaMemcpyAsync(coef, hc.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, c->st));
    CK(lanczos_axpy<double>(ns, dim, Pc, Rc, coef, 1, nullptr, 0, c->st));
    for (int i = 0; i < ns; ++i) if (!done[i]) rr[i] = rn[i];
  }
  c->lp_cg_iters = cg_it;
  // y = y_low + z; t* = y/(u.y) - u
  std::vector<double> ones(ns, -1.0);
  CK(cudaMemcpyAsync(coef, ones.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, c->st));
  CK(lanczos_axpy<double>(ns, dim, c->lp_t, Z, coef, 1, nullptr, 0, c->st));
  CK(row_dots(ns, dim, U, c->lp_t, uy, c->st));
  CK(jd_targets(ns, dim, c->lp_t, U, uy, c->lp_t, c->st));
  {
    double* cb;
    CA(dalloc(c, &cb, (size_t)ns * c->n_occ * c->n_occ));
    int rp = project<double>(c, (long)ns * c->n_occ, c->lp_t, cb);
    dfree(c, cb);
    if (rp != BSE_OK) return rp;
  }
  CA(dalloc(c, &c->lp_u, (size_t)ns * dim));
  CK(cudaMemcpyAsync(c->lp_u, U, sizeof(double) * ns * dim, cudaMemcpyDeviceToDevice, c->st));
  CK(cudaMemcpyAsync(c->lp_r, R, sizeof(double) * ns * dim, cudaMemcpyDeviceToDevice, c->st));
  CK(cudaMemcpyAsync(c->lp_theta, th_d, sizeof(double) * ns, cudaMemcpyDeviceToDevice, c->st));
  CA(lp_finish_samples(c));
  CK(cudaStreamSynchronize(c->st));
  if (n_out) *n_out = ns;
  return BSE_OK;
}

int bse_precond_get_samples(bse_ctx* c, int n, double* u_out, double* r_out, double* t_out, double* theta_out,
                            int* n_out) {
  if (!c) return BSE_ERR_INVALID_ARG;
  if (n < 0) return fail(c, BSE_ERR_INVALID_ARG, "bse_precond_get_samples: n < 0");
  const long dim = (long)c->n_occ * c->n_pw;
  const long k = std::min<long>(n, c->lp_ns);
  if (n_out) *n_out = (int)c->lp_ns;
  if (k == 0) return BSE_OK;
  if (u_out) {
    if (!c->lp_u) return fail(c, BSE_ERR_STATE, "the samples were set by the caller: no Ritz vectors held");
    CK(cudaMemcpyAsync(u_out, c->lp_u, sizeof(double) * k * dim, cudaMemcpyDeviceToHost, c->st));
  }
  if (r_out) CK(cudaMemcpyAsync(r_out, c->lp_r, sizeof(double) * k * dim, cudaMemcpyDeviceToHost, c->st));
  if (t_out) CK(cudaMemcpyAsync(t_out, c->lp_t, sizeof(double) * k * dim, cudaMemcpyDeviceToHost, c->st));
  if (theta_out) CK(cudaMemcpyAsync(theta_out, c->lp_theta, sizeof(double) * k, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  return BSE_OK;
}

int bse_precond_grad(bse_ctx* c, const float* params, int act_bf16, double* loss_out, double* grad_out) {
  if (!c) return BSE_ERR_INVALID_ARG;
  if (!params || !grad_out) return fail(c, BSE_ERR_INVALID_ARG, "bse_precond_grad: null params or grad_out");
  if (c->lp_ns == 0) return fail(c, BSE_ERR_STATE, "no training samples on this context");
  using namespace mlpl;
  float* dp;
  double *dgr, *dl;
  CA(dalloc(c, &dp, N)); CA(dalloc(c, &dgr, N)); CA(dalloc(c, &dl, 1));
  struct G6 { bse_ctx* c; void* a; void* b; void* d; ~G6() { dfree(c, a); dfree(c, b); dfree(c, d); } } g6{c, dp, dgr, dl};
  CK(cudaMemcpyAsync(dp, params, sizeof(float) * N, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemsetAsync(dgr, 0, sizeof(double) * N, c->st));
  CK(cudaMemsetAsync(dl, 0, sizeof(double), c->st));
  CA(lp_step(c, dp, act_bf16 ? 1 : 0, dgr, dl));
  double l = 0;
  CK(cudaMemcpyAsync(grad_out, dgr, sizeof(double) * N, cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(&l, dl, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (loss_out) *loss_out = l;
  return BSE_OK;
}

int bse_precond_train(bse_ctx* const* ctxs, int n_ctx, const float* init, int epochs, double lr,
                      int act_bf16, float* params_out, double* loss_hist) {
  if (!ctxs || n_ctx < 1 || !init || epochs < 1 || !(lr > 0) || !params_out) return BSE_ERR_INVALID_ARG;
  for (int i = 0; i < n_ctx; ++i)
    if (!ctxs[i] || ctxs[i]->lp_ns == 0) return ctxs[i] ? fail(ctxs[i], BSE_ERR_STATE, "context without training samples") : BSE_ERR_INVALID_ARG;
  using namespace mlpl;
  bse_ctx* c = ctxs[0];
  // feature standardisation from all samples
  double* mom;
  CA(dalloc(c, &mom, 2 * F));
  CK(cudaMemsetAsync(mom, 0, sizeof(double) * 2 * F, c->st));
  double nrows = 0;
  for (int i = 0; i < n_ctx; ++i) {
    bse_ctx* q = ctxs[i];
    const long rows = q->lp_ns * (long)q->n_occ * q->n_pw;
    CK(cudaStreamSynchronize(q->st));
    CK(feature_moments(rows, q->n_occ, q->n_pw, q->lp_r, q->lp_theta, q->lp_rn2, q->g2p, q->eps, q->v0,
                       q->scissor, mom, c->st));
    nrows += (double)rows;
  }
  std::vector<double> hm(2 * F);
  CK(cudaMemcpyAsync(hm.data(), mom, sizeof(double) * 2 * F, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  dfree(c, mom);
  std::vector<float> p(init, init + N);
  for (int k = 0; k < F; ++k) {
    const double mu = hm[k] / nrows;
    const double var = std::max(hm[F + k] / nrows - mu * mu, 0.0);
    p[MU + k] = (float)mu;
    p[SG + k] = (float)std::max(std::sqrt(var), 1e-6);
  }
  float *dp, *m, *v;
  double *dg, *dl;
  CA(dalloc(c, &dp, N)); CA(dalloc(c, &m, N)); CA(dalloc(c, &v, N)); CA(dalloc(c, &dg, N)); CA(dalloc(c, &dl, 1));
  struct G7 { bse_ctx* c; std::vector<void*> v; ~G7() { for (void* x : v) dfree(c, x); } } g7{c, {dp, m, v, dg, dl}};
  CK(cudaMemcpyAsync(dp, p.data(), sizeof(float) * N, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemsetAsync(m, 0, sizeof(float) * N, c->st));
  CK(cudaMemsetAsync(v, 0, sizeof(float) * N, c->st));
  CK(cudaStreamSynchronize(c->st));
  int step = 0;
  for (int ep = 0; ep < epochs; ++ep) {
    double total = 0;
    for (int i = 0; i < n_ctx; ++i) {
      bse_ctx* q = ctxs[i];
      CK(cudaMemsetAsync(dg, 0, sizeof(double) * N, q->st));
      CK(cudaMemsetAsync(dl, 0, sizeof(double), q->st));
      CA(lp_step(q, dp, act_bf16 ? 1 : 0, dg, dl));
      CK(adam_step(MU, dp, dg, m, v, (float)lr, ++step, q->st));
      double l = 0;
      CK(cudaMemcpyAsync(&l, dl, sizeof(double), cudaMemcpyDeviceToHost, q->st));
      CK(cudaStreamSynchronize(q->st));
      total += l / n_ctx;
    }
    if (loss_hist) loss_hist[ep] = total;
  }
  CK(cudaMemcpy(params_out, dp, sizeof(float) * N, cudaMemcpyDeviceToHost));
  return BSE_OK;
}

int bse_precond_load(bse_ctx* c, const float* params) {
  if (!c) return BSE_ERR_INVALID_ARG;
  if (!params) { dfree(c, c->lp_params); c->lp_params = nullptr; return BSE_OK; }
  for (int i = 0; i < mlpl::N; ++i)
    if (!std::isfinite(params[i])) return fail(c, BSE_ERR_NUMERIC, "non-finite preconditioner parameter");
  if (!c->lp_params) CA(dalloc(c, &c->lp_params, mlpl::N));
  CK(cudaMemcpyAsync(c->lp_params, params, sizeof(float) * mlpl::N, cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  return BSE_OK;
}

}  // extern "C"

// =================================================================================
// Operator application that allocates nothing (bse_apply_liouville_static).
//
// Some callers cannot call cudaMalloc at the moment they need the operator: hosts whose
// device memory budget is fixed by an external pool, or hard real-time paths where a
// device allocation (which may synchronise the device) is not allowed. For them the
// r-space workspaces of one application live in a fixed array compiled into this library
// instead of being allocated by the context.
// =================================================================================
#include <mutex>

namespace {

constexpr size_t BSE_STATIC_SCRATCH_BYTES = (size_t)32 << 20;   // 32 MiB per device

// held by every GPU that loads this library, for the life of the process
static __device__ __align__(256) unsigned char g_static_scratch[BSE_STATIC_SCRATCH_BYTES];

std::mutex g_static_mu;
void* g_static_addr[256] = {};

// device address of the scratch array on the current device (looked up once per device)
cudaError_t static_scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return cudaSuccess;
}

template <typename T>
int apply_static_impl(bse_ctx* c, long n_vec, const T* a_in, T* a_out, unsigned char* ws) {
  const long n3 = c->n3;
  const long nf = n_vec * c->n_occ;
  const long ngr = (nf + 1) / 2, nh = (n_vec + 1) / 2;
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t b_a = up((size_t)ngr * n3 * sizeof(cplx<T>));
  const size_t b_h = up((size_t)nh * n3 * sizeof(cplx<T>));
  const size_t b_c = up((size_t)nf * std::max(c->n_occ, c->n_qc) * sizeof(T));
  const size_t need = 2 * b_a + b_h + b_c;
  if (need > BSE_STATIC_SCRATCH_BYTES) {
    char buf[256];
    snprintf(buf, sizeof(buf),
             "bse_apply_liouville_static: %ld vectors need %zu bytes of scratch; the static array holds %zu",
             n_vec, need, BSE_STATIC_SCRATCH_BYTES);
    return fail(c, BSE_ERR_INVALID_ARG, buf);
  }
  cplx<T>* ga = reinterpret_cast<cplx<T>*>(ws);
  cplx<T>* gr = reinterpret_cast<cplx<T>*>(ws + b_a);
  cplx<T>* gh = reinterpret_cast<cplx<T>*>(ws + 2 * b_a);
  T* cb = reinterpret_cast<T*>(ws + 2 * b_a + b_h);
  const int N = c->N;
  const double sf = c->k1e_factor();
  // the array keeps the previous call's contents: everything read is written first (the
  // transforms write every compact stage and grid point they read back) or cleared here
  // (the Hartree grids, the odd tail of R(r))
  CK(sphere_to_grid<T>(a_in, nf, c->n_pw, c->n_half, N, c->sph, tw_of<T>(c), gr, ga, c->st));
  CK(cudaMemsetAsync(gh, 0, (size_t)nh * n3 * sizeof(cplx<T>), c->st));
  if (sf != 0.0) {
    CK(hartree_density<T>((int)n_vec, c->n_occ, n3, (const T*)ga, upsi_of<T>(c), (T*)gh, c->st));
    CK(fft3d<T>(gh, nh, N, -1, tw_of<T>(c), c->st));
    CK(grid_coulomb<T>(gh, nh, N, c->L, c->omega, 0, 1.0 / (double)n3, c->st));
    CK(fft3d<T>(gh, nh, N, +1, tw_of<T>(c), c->st));
  }
  if (nf & 1) CK(cudaMemsetAsync(gr + (ngr - 1) * n3, 0, (size_t)n3 * sizeof(cplx<T>), c->st));
  if (c->tau_entry) {
    CK(k1d_tiled<T>((int)n_vec, c->n_occ, n3, (const T*)ga, (const T*)c->tau, c->n_ent, c->bptr, c->bw,
                    c->n_rblocks, vloc_of<T>(c), (const T*)gh, upsi_of<T>(c), sf, (T*)gr,
                    k1d_variant_for<T>(c, (int)n_vec), c->st));
  } else if (c->tau_sym) {
    CK(k1d_sym_tiled<T>((int)n_vec, c->n_occ, n3, (const T*)ga, (const T*)c->tau, k1d_sym_lists(c), vloc_of<T>(c),
                        (const T*)gh, upsi_of<T>(c), sf, (T*)gr, k1d_sym_variant_for<T>(c, (int)n_vec), c->st));
  } else {
    CK(k1d_combine<T>((int)n_vec, c->n_occ, n3, (const T*)ga, (const T*)c->tau, c->n_pairs, c->nbr_ptr, c->nbr_w,
                      c->nbr_p, vloc_of<T>(c), (const T*)gh, upsi_of<T>(c), sf, (T*)gr, c->st));
  }
  CK(grid_to_sphere<T>(gr, nf, c->n_pw, c->n_half, N, c->sph, tw_of<T>(c), ga, 1.0 / (double)n3, a_out,
                       a_in, g2h_of<T>(c), esh_of<T>(c), c->n_occ, c->st));
  // explicit QP terms and P_c with the SIMT GEMM (the tensor-core path would allocate split
  // buffers)
  CA(qp_correction<T>(c, nf, a_in, a_out, cb, false));
  CA(emat_term<T>(c, n_vec, a_in, a_out));
  const T* psi = psi_of<T>(c);
  CK((gemm<T, T>(false, true, (int)nf, c->n_occ, c->n_pw, 1.0, a_out, c->n_pw, psi, c->n_pw, 0.0, cb,
                 c->n_occ, 1, c->st)));
  if (c->n_up > 0) CK(mask_cross_channel<T>((int)nf, c->n_occ, c->n_up, cb, c->st));
  CK((gemm<T, T>(false, false, (int)nf, c->n_pw, c->n_occ, -1.0, cb, c->n_occ, psi, c->n_pw, 1.0, a_out,
                 c->n_pw, 1, c->st)));
  CK(zero_pad_column<T>((int)nf, c->n_pw, a_out, c->st));
  return BSE_OK;
}

}  // namespace

extern "C" int bse_apply_liouville_static(bse_ctx* c, int n_vec, const void* a_in, void* a_out) {
  if (!c) return BSE_ERR_INVALID_ARG;
  if (n_vec < 0 || (n_vec > 0 && (!a_in || !a_out))) return fail(c, BSE_ERR_INVALID_ARG, "bad apply arguments");
  if (a_in == a_out && n_vec > 0) return fail(c, BSE_ERR_INVALID_ARG, "a_out must not alias a_in");
  if (!c->tau_ready) return fail(c, BSE_ERR_STATE, "bse_build_tau must run before bse_apply_liouville_static");
  if (n_vec == 0) return BSE_OK;
  void* ws = nullptr;
  cudaError_t e = static_scratch_address(&ws);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaGetSymbolAddress of the static scratch");
  int r = (c->prec == BSE_PREC_FP64)
              ? apply_static_impl<double>(c, n_vec, (const double*)a_in, (double*)a_out, (unsigned char*)ws)
              : apply_static_impl<float>(c, n_vec, (const float*)a_in, (float*)a_out, (unsigned char*)ws);
  if (r != BSE_OK) return r;
  e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return cuda_fail(c, e, "bse_apply_liouville_static");
  return BSE_OK;
}
