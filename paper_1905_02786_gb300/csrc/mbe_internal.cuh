// Internal declarations shared by the CUDA translation units of libmbe.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>
#include <array>
#include <map>
#include <memory>
#include <unordered_map>
#include <mutex>
#include "../../include/mbe.h"

#define MBE_MAX_ACT 30      // active orbitals per CASCI (string masks are uint32)
#define MBE_MAX_NORB 128    // tuple keys are 128-bit orbital sets
#define MBE_MAX_ORDER 16    // increments enumerate 2^order - 2 subtuples
#define MBE_MAX_DEVICES 64  // per-device one-time set-up flags (mbe_create checks)

// ---------------------------------------------------------------- errors
struct MbeError {
  int code;
  std::string msg;
};

#define CU_CHECK(call)                                                      \
  do {                                                                      \
    cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess)                                                  \
      throw MbeError{MBE_ECUDA, std::string(#call) + ": " +                 \
                                    cudaGetErrorString(e_)};                \
  } while (0)

// Runs f() once per device for the flag array `done` (a kernel attribute, a
// constant table): the check and the set-up are serialised by one mutex per
// call site, so that contexts on several host threads may race to it.
template <class F>
void once_per_device(bool (&done)[MBE_MAX_DEVICES], int device, F f) {
  static std::mutex mu;
  if (device < 0 || device >= MBE_MAX_DEVICES)
    throw MbeError{MBE_EINVAL, "device index out of range"};
  std::lock_guard<std::mutex> lk(mu);
  if (done[device]) return;
  f();
  done[device] = true;
}

// every launch site checks the launch and counts it: g_mbe_launches counts
// kernels run on the device, g_mbe_host_launches the launch calls the host
// makes (a replayed CUDA graph is one).  While this thread captures a graph
// (GraphRunner) the launches are counted into t_capture_kernels instead and
// added to g_mbe_launches each time the graph is launched.
extern int64_t g_mbe_launches;
extern int64_t g_mbe_host_launches;
extern thread_local bool t_capturing;
extern thread_local int64_t t_capture_kernels;
#define CU_LAUNCH_CHECK()                                          \
  do {                                                             \
    if (t_capturing) {                                             \
      t_capture_kernels++;                                         \
    } else {                                                       \
      __atomic_add_fetch(&g_mbe_launches, 1, __ATOMIC_RELAXED);      \
      __atomic_add_fetch(&g_mbe_host_launches, 1, __ATOMIC_RELAXED); \
    }                                                              \
    CU_CHECK(cudaGetLastError());                                  \
  } while (0)

// a CUDA event recorded on s; inside a stream capture it becomes an event
// record node of the graph (recorded each time the graph runs)
inline void record_event(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  if (cs == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  else
    cudaEventRecord(e, s);
}

// CUDA-event timing of the dominant (sigma contraction) kernel
struct KernelTimer {
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
  double ms = 0.0;
  void begin(cudaStream_t s, bool on, cudaEvent_t* a) {
    *a = nullptr;
    if (!on) return;
    cudaEventCreate(a);
    record_event(*a, s);
  }
  void end(cudaStream_t s, cudaEvent_t a) {
    if (!a) return;
    cudaEvent_t b;
    cudaEventCreate(&b);
    record_event(b, s);
    pending.emplace_back(a, b);
  }
  void resolve() {
    for (auto& p : pending) {
      float t = 0.f;
      cudaEventSynchronize(p.second);
      cudaEventElapsedTime(&t, p.first, p.second);
      ms += t;
      cudaEventDestroy(p.first);
      cudaEventDestroy(p.second);
    }
    pending.clear();
  }
};

// ------------------------------------------------- packed symmetric vectors
// The mixed Davidson keeps its FP32 vectors of a closed-shell M_s = 0 space
// (c(a, b) = c(b, a)) packed: the nstr diagonal elements first, padded to
// sym_nd = nstr rounded up to 4, then the strictly upper triangle row by row;
// sym_len elements in all (a multiple of 4, the padding zero).  A dot
// product of two such vectors weighs the upper elements by 2, so it equals
// the dot product of the full vectors.
__host__ __device__ inline int sym_nd(int nstr) { return (nstr + 3) & ~3; }
__host__ __device__ inline int64_t sym_len(int nstr) {
  return ((int64_t)sym_nd(nstr) + (int64_t)nstr * (nstr - 1) / 2 + 3) & ~(int64_t)3;
}
// packed position of element (a, b) or (b, a)
__host__ __device__ inline int64_t sym_index(int a, int b, int nstr) {
  if (a > b) {
    const int t = a;
    a = b;
    b = t;
  }
  return a == b ? (int64_t)a
                : (int64_t)sym_nd(nstr) + (int64_t)a * (2 * nstr - a - 1) / 2 + (b - a - 1);
}

// ------------------------------------------------------------ CUDA graphs
// Replays a launch sequence as one CUDA graph.  run(key, issue) records the
// launches issue() makes on the stream (stream capture), brings the
// executable graph kept for `key` up to date with them (cudaGraphExecUpdate
// sets kernel arguments, grid shapes and events in place; a sequence of
// another shape is instantiated anew) and launches it: one host launch for
// the sequence, its kernels back to back on the device.  issue() must not
// synchronise with the host (the capture fails with an error if it does).
struct GraphRunner {
  cudaStream_t st = nullptr;
  std::map<int, cudaGraphExec_t> exec;
  int64_t instantiated = 0, updated = 0, launched = 0;
  explicit GraphRunner(cudaStream_t s) : st(s) {}
  GraphRunner(const GraphRunner&) = delete;
  GraphRunner& operator=(const GraphRunner&) = delete;
  ~GraphRunner() {
    for (auto& e : exec) cudaGraphExecDestroy(e.second);
  }
  template <class F>
  void run(int key, F issue) {
    CU_CHECK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    t_capturing = true;
    t_capture_kernels = 0;
    cudaGraph_t g = nullptr;
    try {
      issue();
    } catch (...) {
      t_capturing = false;
      cudaStreamEndCapture(st, &g);
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      throw;
    }
    t_capturing = false;
    const int64_t nk = t_capture_kernels;
    CU_CHECK(cudaStreamEndCapture(st, &g));
    auto it = exec.find(key);
    bool ok = false;
    if (it != exec.end()) {
      cudaGraphExecUpdateResultInfo info;
      if (cudaGraphExecUpdate(it->second, g, &info) == cudaSuccess) {
        ok = true;
        updated++;
      } else {
        cudaGetLastError();       // the update's error is not sticky
        cudaGraphExecDestroy(it->second);
        exec.erase(it);
      }
    }
    if (!ok) {
      cudaGraphExec_t e = nullptr;
      const cudaError_t r = cudaGraphInstantiate(&e, g, 0);
      if (r != cudaSuccess) {
        cudaGraphDestroy(g);
        throw MbeError{MBE_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(r)};
      }
      exec[key] = e;
      instantiated++;
    }
    cudaGraphDestroy(g);
    CU_CHECK(cudaGraphLaunch(exec[key], st));
    launched++;
    __atomic_add_fetch(&g_mbe_launches, nk, __ATOMIC_RELAXED);
    __atomic_add_fetch(&g_mbe_host_launches, 1, __ATOMIC_RELAXED);
  }
};

// --------------------------------------------------------- device memory
// A caching allocator: freed blocks are kept per size and reused; the total
// held by the context is capped by mem_cap (0 = no cap).
struct DevPool {
  int64_t cap = 0, held = 0;
  std::multimap<size_t, void*> free_blocks;
  std::unordered_map<void*, size_t> sizes;
  void* alloc(size_t bytes);
  void release(void* p);
  void trim();
  int64_t cached() const;   // bytes held in free blocks (reusable)
  ~DevPool();
};

template <typename T>
struct DevBuf {
  DevPool* pool = nullptr;
  T* ptr = nullptr;
  size_t n = 0;
  DevBuf() {}
  DevBuf(DevPool* p, size_t count) { reset(p, count); }
  void reset(DevPool* p, size_t count) {
    release();
    pool = p;
    n = count;
    ptr = count ? (T*)p->alloc(count * sizeof(T)) : nullptr;
  }
  void release() {
    if (ptr && pool) pool->release(ptr);
    ptr = nullptr;
    n = 0;
  }
  ~DevBuf() { release(); }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
};

// --------------------------------------------------------- string tables
// Strings of nsig electrons in n active orbitals, ordered by the integer
// value of their occupation bit mask (colexicographic rank).  For every
// string I and packed orbital pair P = (p >= q) the table holds the unique
// string J with <I| E_pq + E_qp |J> != 0 (E_pp for p == q) and its sign,
// packed as (J << 1) | (sign < 0), or -1 if there is none.
struct StringTables {
  int n = 0, nsig = 0, nstr = 0, npair = 0;
  DevBuf<uint32_t> masks;  // nstr
  DevBuf<int32_t> link;    // nstr * npair
  // the same links compacted per string (tensor-core sigma, built on first
  // use): nlink = nsig (n - nsig + 1) entries (J << 8) | (P << 1) | (sign < 0)
  // per string, ascending in P
  DevBuf<int32_t> lnk;
  int nlink = -1;
  // for every string J its links ordered by the 128-string tile of the
  // linked string, as offsets into the tensor-core sigma's staged tile
  // (plist, int16 with the sign in bit 15) and the first entry of each tile
  // (poff, ntiles + 1 per string)
  DevBuf<int16_t> plist;
  DevBuf<int32_t> poff;
};

// ------------------------------------------------------------- context
// Spin-summed active-space RDMs of one converged CASCI, kept on the device
// for the energy backward (keep_ci): gamma+_P = <c|E+_P|c> for the npair
// packed pairs, then the upper triangle (P <= Q, row by row) of
// Gamma'_PQ = <E+_P c, E+_Q c>, both for the normalised vector.
struct KeptRdm {
  int order;
  std::vector<int32_t> tuple;  // global orbital ids of the tuple
  int n, nsig;
  const double* rdm = nullptr; // rdm_size(npair) doubles inside a RdmBlock
};
struct RdmBlock {
  int order;
  std::unique_ptr<DevBuf<double>> buf;
};
inline int64_t rdm_size(int npair) { return npair + (int64_t)npair * (npair + 1) / 2; }
// packed RDMs (rdm_size(tab->npair) doubles per vector, into out) of the B
// converged vectors X (B * nstr_alpha * nstr_beta, FP64; alpha strings tab,
// beta strings tabb); fp32: products and the sums inside a tile in FP32
// (vectors of the mixed path), else FP64 throughout
void rdm_batch(mbe_ctx* ctx, const StringTables* tab, const StringTables* tabb, const double* X,
               int B, bool fp32, double* out);

struct HashTable {
  int64_t cap = 0;             // power of two
  int64_t count = 0;
  DevBuf<unsigned long long> keys;  // 2 words per slot
  DevBuf<double> val;          // increment
  DevBuf<uint8_t> keep;        // screening flag
  DevBuf<int32_t> state;       // 0 empty, 1 claimed/filled
};

// Warm starts: the converged CI vectors (FP32) of the tuples solved at one
// order, keyed by tuple (128-bit orbital set); a tuple of the next order
// starts its Davidson iteration from a parent's vector with the added
// orbital inserted (empty, or doubly occupied with its fermion sign).
struct KeyHash {
  size_t operator()(const std::pair<uint64_t, uint64_t>& k) const {
    return (size_t)(k.first * 0x9E3779B97F4A7C15ull ^ (k.second + 0x632BE59BD9B4E019ull +
                                                         (k.first << 6) + (k.first >> 2)));
  }
};
struct GuessStore {
  int order = -1;
  std::vector<std::unique_ptr<DevBuf<float>>> blocks;
  std::unordered_map<std::pair<uint64_t, uint64_t>, const float*, KeyHash> map;
  int64_t bytes = 0;
  void clear() {
    map.clear();
    blocks.clear();
    bytes = 0;
    order = -1;
  }
};
// tuples b of a batch that start from a parent vector src, the added
// orbital at active position jo, occupied (occ = 1) or empty
struct GuessPlan {
  std::vector<int32_t> b, jo, occ;
  std::vector<const float*> src;
};

struct OrderRec {
  int order;
  std::vector<int32_t> tuples;   // ntup * order
  std::vector<double> eps, inc;
  std::vector<uint8_t> keep;
};

struct mbe_ctx {
  int device = 0;
  mbe_stats stats = {};
  int64_t launch_base = 0, host_launch_base = 0;
  KernelTimer dom_timer;     // tensor-core sigma launches
  KernelTimer fp64_timer;    // FP64 contraction launches
  mbe_options opt;
  cudaStream_t stream = nullptr;      // stream all work is issued on
  cudaStream_t own_stream = nullptr;  // the context's own stream
  std::string last_error;
  DevPool pool;

  // integrals
  // nocc: doubly occupied orbitals of the reference determinant (the beta
  // occupation); nocc_a = nocc + two_sz: alpha occupation (high spin)
  int norb = 0, nelec = 0, nocc = 0, npair_g = 0, nocc_a = 0, two_sz = 0;
  DevBuf<double> h, eri;
  std::vector<double> h_host, eri_host;

  // reference / expansion space
  std::vector<int> ref, exp;
  bool have_ref = false;
  double e_ref = 0.0;

  // string tables per (n, nsig)
  std::map<std::pair<int, int>, StringTables*> tables;

  // MBE state
  HashTable hash;
  int last_order = 0;                 // highest order with increments
  int cur_order = 0;                  // order of the last solved tuples
  std::vector<int32_t> cur_tuples;    // ntup * cur_order (host)
  std::vector<double> cur_eps;
  DevBuf<int32_t> cur_tuples_dev;
  DevBuf<double> cur_eps_dev;
  std::vector<int32_t> prev_tuples;   // last processed order (host)
  std::vector<uint8_t> prev_keep;
  int prev_order = 0;
  std::vector<double> order_sums;
  std::vector<OrderRec> history;      // every processed order
  // all solved tuples (for the backward): order, tuple, kept RDMs
  std::vector<KeptRdm> kept;
  bool kept_ref = false;
  KeptRdm ref_ci;
  std::vector<RdmBlock> rdm_blocks;
  // autotuned operand plans of the two-spin tensor-core sigma:
  // (n, nsig) -> {A stages, pull lists in shared memory, epilogue groups};
  // tune_file is the cache (empty: none)
  std::map<std::pair<int, int>, std::array<int, 3>> tune_ab;
  std::string tune_file;
  // warm-start vectors of the previous and the current order
  GuessStore guess_prev, guess_cur;
  // pi-pruning: partner[o] = the degenerate partner of expansion orbital o
  // (-1 if none); tuples are unions of units (single orbitals and pairs)
  bool pruned = false;
  std::vector<int32_t> partner;
  DevBuf<int32_t> partner_dev;

  ~mbe_ctx();
};

// ------------------------------------------------- per-bin solver state
struct BinProblem {
  int n, nsig, nstr, npair;      // nsig, nstr: alpha electrons and strings
  int nsigb = -1, nstrb = -1;    // beta electrons and strings
  int64_t ndet;                  // nstr * nstrb
  int B;                         // tuples in this batch
  const StringTables* tab;       // alpha strings
  const StringTables* tabb = nullptr;   // beta strings (== tab for a closed shell)
  bool closed() const { return tabb == tab; }
  // Ms(Ms+1) of every determinant of the space, Ms = (nsig - nsigb) / 2
  double msms() const { return 0.25 * (nsig - nsigb) * (nsig - nsigb + 2); }
  // beta side = alpha side (closed shell)
  void set_closed() {
    nsigb = nsig;
    nstrb = nstr;
    tabb = tab;
  }
  DevBuf<int32_t> act;           // B * n global orbital ids
  DevBuf<double> ecore;          // B
  DevBuf<double> heff;           // B * n * n
  DevBuf<double> hp;             // B * n * n   (h' = heff - 1/2 sum_r (pr|rq))
  DevBuf<double> gp;             // B * npair * npair
  DevBuf<double> jk;             // B * 2 * n * n  (J_pq = (pp|qq), K_pq = (pq|qp))
  DevBuf<uint8_t> gsplit;        // g'/2 as bf16 hi/lo rows (tensor-core sigma operand source)
  DevBuf<uint8_t> haa;           // one-spin Hamiltonian H^alpha as bf16 hi/lo rows
};

// P-space preconditioner of the mixed Davidson iteration (mbe_pspace.cu):
// per tuple the npp lowest-diagonal symmetric basis functions, the
// eigenvectors U and eigenvalues of A restricted to them
struct PspaceWork {
  int npp = 0;
  DevBuf<int32_t> sel;   // B * 128 canonical determinant indices
  DevBuf<float> lam;     // B * 128
  DevBuf<float> U;       // B * 128 * 128
};
// the P-space size used for a bin (0: off) given the requested size
int pspace_size(const BinProblem& bp, int requested);
// hd, T, V, Uo, X: one vector per tuple every ld elements
void pspace_setup(mbe_ctx* ctx, BinProblem& bp, const float* hd, int64_t ld, double shift,
                  int npp, PspaceWork& w);
// the P-space block of t (and with olsen of u = M^-1 x in Uo, X the Ritz
// vector), correcting the partial dot products that the residual kernel left
void pspace_apply(mbe_ctx* ctx, const BinProblem& bp, const PspaceWork& w, float* T,
                  const float* hd, int64_t ld, const double* theta, const float* V, int m, int M,
                  int nchunks, double* partial, bool fix_dots, const int32_t* active,
                  bool olsen, float* Uo, const float* X, double* upart, double* xpart);

// ------------------------------------------------------------ launchers
void build_string_tables(mbe_ctx* ctx, StringTables* t);
// raw-pointer forms of the table, integral and FP64 sigma launchers (they
// allocate nothing)
int64_t string_count(int n, int nsig);
void launch_string_tables(mbe_ctx* ctx, int n, int nsig, int nstr, uint32_t* masks,
                          int32_t* link);
// nel: active electrons (both spins)
void launch_effints_raw(mbe_ctx* ctx, const int32_t* act, int B, int n, int nel, double* ecore,
                        double* heff, double* hp, double* gp, double* jk);
void sigma_fp64_raw(mbe_ctx* ctx, int n, int nsig, int nstr, const int32_t* link,
                    const uint32_t* masks, const double* gp, const double* c, int64_t c_stride,
                    double* out, int64_t out_stride, const int32_t* active, const int32_t* bmap,
                    int nb, double* D, double* E, double spin_shift, bool emulated, int32_t* err,
                    bool symmetric = false, int b_first = 0, int nsigb = -1, int nstrb = -1,
                    const int32_t* linkb = nullptr, const uint32_t* masksb = nullptr);
StringTables* get_tables(mbe_ctx* ctx, int n, int nsig);
// active electrons of each spin: alpha (orbitals below nocc_a), beta (below nocc)
int count_sig(const mbe_ctx* ctx, const std::vector<int>& act);
int count_sig_b(const mbe_ctx* ctx, const std::vector<int>& act);
// D[P][K] = (E+_P c)(K) for one CI vector c (ndet) and every packed pair P
// mbe_sigma_noalloc (scratch in a file-scope device array)
int noalloc_sigma_run(mbe_ctx* ctx, const int* act, int nact, const double* c_dev,
                      double* sigma_dev, int64_t ndet_arg, double* e_core);
// energy gradient of the processed expansion (mbe_energy_backward)
int backward_run(mbe_ctx* ctx, double scale, double* dh_host, double* deri_host);
void launch_effints(mbe_ctx* ctx, BinProblem& bp);
void launch_hdiag(mbe_ctx* ctx, BinProblem& bp, double spin_shift, double* hd);

// sigma for a batch: out[b] = (H_act + shift S^2) c[b] for b < B; c/out with
// strides (elements between consecutive tuples' vectors); active may be NULL.
struct SigmaWork {
  DevBuf<double> D, E;           // scratch for the FP64 path
  DevBuf<float> Xf;              // W rows of the tensor-core path (sigma = W + W^T)
  DevBuf<uint8_t> csplit;        // the vectors as bf16 hi/lo rows (tensor-core operands)
  DevBuf<int32_t> err;           // timeout flag of the tensor-core path
  DevBuf<uint8_t> gex;           // g' digit planes of the fused exact sigma
  DevBuf<int32_t> gexp;          // their row exponents
  DevBuf<float> rmax;            // largest |c| per row (exact sigma's digit scales)
  int64_t sub_batch = 0;
};
bool sigma_tc_supported(int n, int nstr);
// FP32 vectors in and out (c = c^T assumed: sigma = X + X^T)
// packed: c and the result in the packed symmetric layout (sym_index)
void sigma_tc(mbe_ctx* ctx, BinProblem& bp, SigmaWork& w, const float* c, int64_t c_stride,
              float* out, int64_t out_stride, const int32_t* active, double spin_shift,
              bool packed = false);
int32_t sigma_tc_error(mbe_ctx* ctx, SigmaWork& w);
// subspace vectors allocated per tuple by the mixed Davidson: max_subspace
// (clamped to 4..32) for its first stage and its refinement rounds, up to 12
// more (at most 32) for the rounds after one that filled its subspace
inline int mixed_subspace_alloc(int max_subspace) {
  const int ms = max_subspace < 4 ? 4 : (max_subspace > 32 ? 32 : max_subspace);
  return ms + 12 < 32 ? ms + 12 : 32;
}
// Davidson of the mixed-precision mode: FP32 vectors, FP64-grade exact points
void davidson_batch_mixed(mbe_ctx* ctx, BinProblem& bp, double* e_out_host,
                          int32_t* status_host, double* x_out_dev, const GuessPlan* plan);
void convert_f64_to_f32(mbe_ctx* ctx, const double* src, float* dst, int64_t n);
// overwrite the start vectors V[b] (stride vstride) of the planned tuples
// with their parents' vectors (exactly one of V32 / V64 non-null)
void launch_parent_guess(mbe_ctx* ctx, const GuessPlan& plan, int n, int nsig, int nstr,
                         float* V32, double* V64, int64_t vstride);
// emulated: the contraction runs as the FP64-grade sliced tensor-core GEMM
// symmetric: c(a,b) = c(b,a) for every tuple (sigma = X + X^T, coalesced);
// otherwise any c
void sigma_fp64(mbe_ctx* ctx, BinProblem& bp, SigmaWork& w, const double* c,
                int64_t c_stride, double* out, int64_t out_stride,
                const int32_t* active, double spin_shift, bool emulated,
                bool symmetric = false);
bool ozaki_supported(int npair);
// FP64-grade sigma of FP32 vectors c (c = c^T, |c_i| <= 1) fused on the
// tensor cores: writes the rows X (sigma = X + X^T + shift S^2 c follows in
// launch_finish_sym_fp64)
bool sigma_exact_supported(int npair, int nstr);
// the fused exact sigma's one-time set-up of a batch (buffers, g' digit
// planes; sigma_exact makes it on its first call when this was not called)
void sigma_exact_prepare(mbe_ctx* ctx, BinProblem& bp, SigmaWork& w);
void sigma_exact(mbe_ctx* ctx, BinProblem& bp, SigmaWork& w, const float* c, int64_t c_stride,
                 double* X, int64_t x_stride, const int32_t* active);
// out = X + X^T + shift S^2 c in place for every tuple of the batch (c = c^T)
void launch_finish_sym_fp64(mbe_ctx* ctx, const BinProblem& bp, double* out, int64_t out_stride,
                            const double* c, int64_t c_stride, double spin_shift,
                            const int32_t* active);
void contract_ozaki(mbe_ctx* ctx, const double* gp, int npair, const double* D, int64_t ndet,
                    int nb, const int32_t* active, const int32_t* bmap, double* E,
                    int32_t* err);
void s2_apply(mbe_ctx* ctx, BinProblem& bp, const double* c, int64_t c_stride,
              double* out, int64_t out_stride, const int32_t* active);

// Davidson for a batch; writes e_out (B, total energies incl. core),
// status (B), s2 (B), and, if x_out != NULL, the converged vectors (B*ndet).
void davidson_batch(mbe_ctx* ctx, BinProblem& bp, double* e_out_host,
                    int32_t* status_host, double* s2_host, double* x_out_dev,
                    const GuessPlan* plan = nullptr);

// hash / increments
void hash_init(mbe_ctx* ctx, int64_t cap);
void hash_insert(mbe_ctx* ctx, const int32_t* tuples_dev, int order, int64_t ntup,
                 const double* vals_dev, const uint8_t* keep_dev);
void increments_kernel_launch(mbe_ctx* ctx, const int32_t* tuples_dev, int order,
                              int64_t ntup, const double* eps_dev, double eps_ref,
                              double thr, double* inc_dev, uint8_t* keep_dev,
                              int32_t* err_dev);
double kahan_sum_device(mbe_ctx* ctx, const double* v, int64_t n);
// adds the MBE coefficient contributions of one order's tuples to coef (per
// hash slot) and coef_ref (the empty tuple)
void mbe_coef_launch(mbe_ctx* ctx, const int32_t* tuples_dev, int order, int64_t ntup,
                     int32_t* coef_dev, int32_t* coef_ref_dev, int32_t* err_dev);
// tuples of order k of a pi-pruned expansion (host rows, lexicographic)
std::vector<int32_t> next_tuples_pruned(mbe_ctx* ctx, int k);
int64_t next_tuples_device(mbe_ctx* ctx, const int32_t* parents_dev, int order_prev,
                           int64_t nparents, const int32_t* exp_dev, int nexp,
                           DevBuf<int32_t>& out);
