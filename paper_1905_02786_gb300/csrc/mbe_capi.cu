// C ABI of libmbe (declared in include/mbe.h): context, integrals, reference
// space, batched CASCI solves, increments, tuple generation, gradient.
#include "mbe_internal.cuh"
#include <tuple>
#include <fstream>
#include <sstream>
#include <algorithm>
#include <cmath>
#include <cstring>
#include <set>

int64_t g_mbe_launches = 0;
int64_t g_mbe_host_launches = 0;
thread_local bool t_capturing = false;
thread_local int64_t t_capture_kernels = 0;

// ------------------------------------------------------------ DevPool
void* DevPool::alloc(size_t bytes) {
  if (bytes == 0) return nullptr;
  bytes = (bytes + 255) & ~(size_t)255;
  auto it = free_blocks.lower_bound(bytes);
  if (it != free_blocks.end() && it->first <= bytes + bytes / 4) {
    void* p = it->second;
    free_blocks.erase(it);
    return p;
  }
  if (cap > 0 && held + (int64_t)bytes > cap) {
    trim();
    if (held + (int64_t)bytes > cap)
      throw MbeError{MBE_ENOMEM, "device memory cap exceeded (" + std::to_string(bytes) +
                                     " bytes requested)"};
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    trim();
    e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw MbeError{MBE_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed"};
    }
  }
  sizes[p] = bytes;
  held += bytes;
  return p;
}

void DevPool::release(void* p) {
  if (!p) return;
  auto it = sizes.find(p);
  if (it == sizes.end()) return;
  free_blocks.emplace(it->second, p);
}

void DevPool::trim() {
  if (free_blocks.empty()) return;
  cudaDeviceSynchronize();
  for (auto& kv : free_blocks) {
    cudaFree(kv.second);
    held -= sizes[kv.second];
    sizes.erase(kv.second);
  }
  free_blocks.clear();
}

int64_t DevPool::cached() const {
  int64_t t = 0;
  for (const auto& kv : free_blocks) t += (int64_t)kv.first;
  return t;
}

DevPool::~DevPool() {
  cudaDeviceSynchronize();
  for (auto& kv : sizes) cudaFree(kv.first);
}

mbe_ctx::~mbe_ctx() {
  for (auto& kv : tables) delete kv.second;
  tables.clear();
}

// ------------------------------------------------------------ helpers
namespace {

int fail(mbe_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  return code;
}

template <typename F>
int guarded(mbe_ctx* ctx, F&& f) {
  if (!ctx) return MBE_EINVAL;
  try {
    CU_CHECK(cudaSetDevice(ctx->device));
    int r = f();
    if (r == MBE_OK) ctx->last_error.clear();
    return r;
  } catch (const MbeError& e) {
    cudaGetLastError();
    return fail(ctx, e.code, e.msg);
  } catch (const std::bad_alloc&) {
    return fail(ctx, MBE_ENOMEM, "host allocation failed");
  }
}

}  // namespace

StringTables* get_tables(mbe_ctx* ctx, int n, int nsig) {
  auto key = std::make_pair(n, nsig);
  auto it = ctx->tables.find(key);
  if (it != ctx->tables.end()) return it->second;
  StringTables* t = new StringTables();
  t->n = n;
  t->nsig = nsig;
  try {
    build_string_tables(ctx, t);
  } catch (...) {
    delete t;
    throw;
  }
  ctx->tables[key] = t;
  return t;
}

int count_sig(const mbe_ctx* ctx, const std::vector<int>& act) {
  int s = 0;
  for (int a : act) s += a < ctx->nocc_a;
  return s;
}

int count_sig_b(const mbe_ctx* ctx, const std::vector<int>& act) {
  int s = 0;
  for (int a : act) s += a < ctx->nocc;
  return s;
}

namespace {

std::pair<uint64_t, uint64_t> orbital_key(const std::vector<int>& orbs) {
  uint64_t k0 = 0, k1 = 0;
  for (int o : orbs) {
    if (o < 64) k0 |= 1ull << o;
    else k1 |= 1ull << (o - 64);
  }
  return {k0, k1};
}

// Solve the CASCI of every active space in `acts` (the tuples of one order,
// or the reference space as order 0); binned by (n, nsig).  With warm starts
// on, a tuple whose parent (the tuple less one orbital) was solved at the
// previous order starts from that vector, and the converged vectors of this
// call are kept for the next order.  With rdm_out the packed RDMs of every
// converged vector are formed on the device right after its batch (blocks
// tagged with the order in ctx->rdm_blocks) and rdm_out[j] points at those
// of acts[j]; no CI vector leaves the device.
void solve_jobs(mbe_ctx* ctx, const std::vector<std::vector<int>>& acts, double* eps,
                int32_t* status, std::vector<const double*>* rdm_out, int order) {
  const bool warm = ctx->opt.warm_start != 0;
  if (warm) {
    if (ctx->guess_cur.order == order - 1) {
      std::swap(ctx->guess_prev, ctx->guess_cur);
      ctx->guess_cur.clear();
    } else if (ctx->guess_cur.order != order) {
      ctx->guess_prev.clear();
      ctx->guess_cur.clear();
    }
    ctx->guess_cur.order = order;
  }
  std::vector<char> is_ref(ctx->norb, 0);
  for (int r : ctx->ref) is_ref[r] = 1;
  // bins: (n, alpha electrons, beta electrons); the two counts differ only
  // for a high-spin reference
  std::map<std::tuple<int, int, int>, std::vector<int64_t>> bins;
  for (int64_t j = 0; j < (int64_t)acts.size(); j++) {
    int n = (int)acts[j].size();
    if (n < 1 || n > MBE_MAX_ACT) throw MbeError{MBE_EINVAL, "active space size out of range"};
    if (n > 15) throw MbeError{MBE_EINVAL, "active spaces above 15 orbitals are not supported"};
    bins[{n, count_sig(ctx, acts[j]), count_sig_b(ctx, acts[j])}].push_back(j);
  }
  if (rdm_out) rdm_out->assign(acts.size(), nullptr);
  size_t free_b = 0, total_b = 0;
  CU_CHECK(cudaMemGetInfo(&free_b, &total_b));
  // the pool's cached free blocks are reusable: they count as free
  double budget = std::min(0.5 * ((double)free_b + (double)ctx->pool.cached()), 96e9);
  if (ctx->opt.mem_cap_bytes > 0) budget = std::min(budget, 0.5 * (double)ctx->opt.mem_cap_bytes);
  const int M = std::max(4, std::min(32, ctx->opt.max_subspace));
  for (auto& kv : bins) {
    const int n = std::get<0>(kv.first), nsig = std::get<1>(kv.first);
    const int nsigb = std::get<2>(kv.first);
    StringTables* tab = get_tables(ctx, n, nsig);
    StringTables* tabb = nsigb == nsig ? tab : get_tables(ctx, n, nsigb);
    const bool closed = tabb == tab;
    const int64_t N = (int64_t)tab->nstr * tabb->nstr;
    // device bytes per tuple: the mixed Davidson holds V and AV (M packed
    // vectors each, N/2 FP32 elements) and five packed FP32 work vectors,
    // the full FP32 exact-point operand, two full FP64 exact-point vectors,
    // the FP32 W rows of the sigma, the bf16 hi/lo copies of the sigma
    // operand and of H^alpha and the P-space eigenvectors; the FP64 one
    // 2M + 6 FP64 vectors
    // the mixed path works on alpha<->beta symmetric vectors: closed shells
    const bool mixed_bin = ctx->opt.precision == MBE_MIXED_BF16X3 && N > 1 && closed &&
                           sigma_tc_supported(n, tab->nstr) && ozaki_supported(tab->npair);
    const int Mm = mixed_subspace_alloc(ctx->opt.max_subspace);
    double per = (mixed_bin ? (double)(4 * Mm + 46) * N + 128.0 * 129.0 * 4.0
                            : (double)(2 * M + 6) * N * 8.0) +
                 (double)tab->npair * tab->npair * 8.0 * 2.0;
    int64_t bmem = std::max<int64_t>(1, (int64_t)(budget / per));
    int64_t bmax = std::min<int64_t>(std::max(1, ctx->opt.max_batch), bmem);
    const std::vector<int64_t>& idx = kv.second;
    for (size_t c0 = 0; c0 < idx.size(); c0 += bmax) {
      const int B = (int)std::min<int64_t>(bmax, (int64_t)idx.size() - (int64_t)c0);
      BinProblem bp;
      bp.n = n;
      bp.nsig = nsig;
      bp.nstr = tab->nstr;
      bp.npair = tab->npair;
      bp.ndet = N;
      bp.B = B;
      bp.tab = tab;
      bp.nsigb = nsigb;
      bp.nstrb = tabb->nstr;
      bp.tabb = tabb;
      std::vector<int32_t> act_h((size_t)B * n);
      for (int b = 0; b < B; b++)
        for (int i = 0; i < n; i++) act_h[(size_t)b * n + i] = acts[idx[c0 + b]][i];
      bp.act.reset(&ctx->pool, act_h.size());
      CU_CHECK(cudaMemcpyAsync(bp.act.ptr, act_h.data(), sizeof(int32_t) * act_h.size(),
                               cudaMemcpyHostToDevice, ctx->stream));
      launch_effints(ctx, bp);
      // warm-start plan: the first parent found in the previous order's store
      // (closed shells: the stored vectors are alpha<->beta symmetric)
      GuessPlan plan;
      if (warm && closed && order >= 1 && ctx->guess_prev.order == order - 1)
        for (int b = 0; b < B; b++) {
          const std::vector<int>& act = acts[idx[c0 + b]];
          std::vector<int> tup;
          for (int o : act)
            if (!is_ref[o]) tup.push_back(o);
          for (int r = (int)tup.size() - 1; r >= 0; r--) {
            std::vector<int> par(tup);
            par.erase(par.begin() + r);
            auto it = ctx->guess_prev.map.find(orbital_key(par));
            if (it == ctx->guess_prev.map.end()) continue;
            const int o = tup[r];
            plan.b.push_back(b);
            plan.jo.push_back((int)(std::lower_bound(act.begin(), act.end(), o) - act.begin()));
            plan.occ.push_back(o < ctx->nocc ? 1 : 0);
            plan.src.push_back(it->second);
            break;
          }
        }
      // keep this batch's vectors for the next order if they fit the cap
      const int64_t keep_bytes = (int64_t)B * N * 4;
      const bool keep =
          warm && closed && ctx->guess_cur.bytes + keep_bytes <= (int64_t)(0.25 * budget);
      DevBuf<double> X;
      if (rdm_out || keep) X.reset(&ctx->pool, (size_t)B * N);
      std::vector<double> e(B);
      std::vector<int32_t> s(B);
      const bool mixed = mixed_bin;
      const GuessPlan* pp = plan.b.empty() ? nullptr : &plan;
      if (mixed)
        davidson_batch_mixed(ctx, bp, e.data(), s.data(), X.ptr, pp);
      else
        davidson_batch(ctx, bp, e.data(), s.data(), nullptr, X.ptr, pp);
      if (keep) {
        auto blk = std::make_unique<DevBuf<float>>(&ctx->pool, (size_t)B * N);
        convert_f64_to_f32(ctx, X.ptr, blk->ptr, (int64_t)B * N);
        for (int b = 0; b < B; b++) {
          const std::vector<int>& act = acts[idx[c0 + b]];
          std::vector<int> tup;
          for (int o : act)
            if (!is_ref[o]) tup.push_back(o);
          ctx->guess_cur.map[orbital_key(tup)] = blk->ptr + (int64_t)b * N;
        }
        ctx->guess_cur.blocks.push_back(std::move(blk));
        ctx->guess_cur.bytes += keep_bytes;
      }
      for (int b = 0; b < B; b++) {
        if (eps) eps[idx[c0 + b]] = e[b];
        if (status) status[idx[c0 + b]] = s[b];
      }
      if (rdm_out) {
        const int64_t rs = rdm_size(tab->npair);
        RdmBlock blk{order, std::make_unique<DevBuf<double>>(&ctx->pool, (size_t)(B * rs))};
        rdm_batch(ctx, tab, tabb, X.ptr, B, mixed, blk.buf->ptr);
        for (int b = 0; b < B; b++) (*rdm_out)[idx[c0 + b]] = blk.buf->ptr + b * rs;
        ctx->rdm_blocks.push_back(std::move(blk));
      }
    }
  }
}

std::vector<int> active_of(const mbe_ctx* ctx, const int32_t* t, int order) {
  std::vector<int> a(ctx->ref.begin(), ctx->ref.end());
  for (int i = 0; i < order; i++) a.push_back(t[i]);
  std::sort(a.begin(), a.end());
  return a;
}

}  // namespace

// ------------------------------------------------------------ C ABI
extern "C" {

void mbe_default_options(mbe_options* o) {
  if (!o) return;
  o->precision = MBE_FP64;
  o->max_batch = 256;
  o->max_subspace = 20;
  o->max_iter = 400;
  o->conv_tol_r = 1e-8;
  o->conv_tol_e = 1e-12;
  o->spin_shift = 0.5;
  o->keep_ci = 0;
  o->deterministic = 1;
  o->mem_cap_bytes = 0;
  o->timing = 0;
  o->verbose = 0;
  o->backward_share = 0;
  o->warm_start = 0;
  o->mixed_stage_tol = 1e-5;
  o->mixed_round_drop = 1e-2;
  o->mixed_rel_tol = 2e-7;
  o->pspace = 128;
  o->wait_limit = 1LL << 24;
  o->autotune = 0;
  o->tune_file = nullptr;
  o->graphs = 1;
}

int mbe_create(mbe_ctx** out, int device, const mbe_options* opt) {
  if (!out) return MBE_EINVAL;
  *out = nullptr;
  mbe_options o;
  mbe_default_options(&o);
  if (opt) o = *opt;
  if (o.precision != MBE_FP64 && o.precision != MBE_MIXED_BF16X3 &&
      o.precision != MBE_EMULATED_FP64)
    return MBE_EINVAL;
  if (o.max_batch < 1 || o.max_subspace < 4 || o.max_subspace > 32 || o.max_iter < 1)
    return MBE_EINVAL;
  if (!(o.mixed_stage_tol > 0.0) || !(o.mixed_round_drop > 0.0 && o.mixed_round_drop < 1.0) ||
      !(o.mixed_rel_tol > 0.0) || o.pspace < 0 || o.pspace > 128 || o.wait_limit < 0 ||
      (o.autotune != 0 && o.autotune != 1) || (o.graphs != 0 && o.graphs != 1))
    return MBE_EINVAL;
  int ndev = 0;
  if (device < 0 || device >= MBE_MAX_DEVICES) return MBE_EINVAL;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device >= ndev) {
    cudaGetLastError();
    return MBE_ECUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return MBE_ECUDA;
  mbe_ctx* c = new mbe_ctx();
  c->device = device;
  c->opt = o;
  c->opt.tune_file = nullptr;   // the caller's string is not kept
  if (o.tune_file) {
    c->tune_file = o.tune_file;
    // cached plans: "sigma_ab n nsig nstages pull_smem groups ms" per line
    std::ifstream in(c->tune_file);
    std::string line;
    while (std::getline(in, line)) {
      std::istringstream ls(line);
      std::string tag;
      int n = 0, ns = 0, nst = 0, ps = 0, ng = 0;
      if (ls >> tag >> n >> ns >> nst >> ps >> ng && tag == "sigma_ab" && nst >= 2 && nst <= 4 &&
          (ps == 0 || ps == 1) && (ng == 1 || ng == 2))
        c->tune_ab[{n, ns}] = {nst, ps, ng};
    }
  }
  c->pool.cap = o.mem_cap_bytes;
  if (cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete c;
    return MBE_ECUDA;
  }
  c->stream = c->own_stream;
  *out = c;
  return MBE_OK;
}

void mbe_destroy(mbe_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  cudaStream_t s = ctx->own_stream;
  delete ctx;
  cudaStreamDestroy(s);
}

int mbe_set_stream(mbe_ctx* ctx, void* stream) {
  return guarded(ctx, [&]() -> int {
    CU_CHECK(cudaStreamSynchronize(ctx->stream));
    ctx->stream = stream ? (cudaStream_t)stream : ctx->own_stream;
    return MBE_OK;
  });
}

const char* mbe_last_error(const mbe_ctx* ctx) {
  return ctx ? ctx->last_error.c_str() : "null context";
}

int mbe_load_integrals(mbe_ctx* ctx, int norb, int nelec, const double* h, const double* eri) {
  return guarded(ctx, [&]() -> int {
    if (norb < 1 || norb > MBE_MAX_NORB) return fail(ctx, MBE_EINVAL, "norb out of range");
    if (nelec < 0 || (nelec + 1) / 2 > norb)
      return fail(ctx, MBE_EINVAL, "nelec must fit the orbitals");
    if (!h || !eri) return fail(ctx, MBE_EINVAL, "null integral pointer");
    const int64_t np = (int64_t)norb * (norb + 1) / 2;
    for (int64_t i = 0; i < (int64_t)norb * norb; i++)
      if (!std::isfinite(h[i])) return fail(ctx, MBE_EINVAL, "non-finite h");
    for (int64_t i = 0; i < np * np; i++)
      if (!std::isfinite(eri[i])) return fail(ctx, MBE_EINVAL, "non-finite eri");
    ctx->norb = norb;
    ctx->nelec = nelec;
    // lowest spin of the high-spin family: singlet or doublet
    ctx->two_sz = nelec % 2;
    ctx->nocc = (nelec - ctx->two_sz) / 2;
    ctx->nocc_a = ctx->nocc + ctx->two_sz;
    ctx->npair_g = (int)np;
    ctx->h_host.assign(h, h + (int64_t)norb * norb);
    ctx->eri_host.assign(eri, eri + np * np);
    ctx->h.reset(&ctx->pool, (size_t)norb * norb);
    ctx->eri.reset(&ctx->pool, (size_t)(np * np));
    CU_CHECK(cudaMemcpyAsync(ctx->h.ptr, h, sizeof(double) * norb * norb, cudaMemcpyHostToDevice,
                             ctx->stream));
    CU_CHECK(cudaMemcpyAsync(ctx->eri.ptr, eri, sizeof(double) * np * np, cudaMemcpyHostToDevice,
                             ctx->stream));
    CU_CHECK(cudaStreamSynchronize(ctx->stream));
    ctx->have_ref = false;
    ctx->kept.clear();
    ctx->kept_ref = false;
    ctx->rdm_blocks.clear();
    ctx->guess_prev.clear();
    ctx->guess_cur.clear();
    ctx->last_order = 0;
    ctx->cur_order = 0;
    ctx->order_sums.clear();
    return MBE_OK;
  });
}

int mbe_set_spin(mbe_ctx* ctx, int two_sz) {
  return guarded(ctx, [&]() -> int {
    if (ctx->norb == 0) return fail(ctx, MBE_ESTATE, "no integrals loaded");
    if (two_sz < 0 || two_sz > ctx->nelec || (ctx->nelec - two_sz) % 2)
      return fail(ctx, MBE_EINVAL, "two_sz must be in 0..nelec with the parity of nelec");
    const int nb = (ctx->nelec - two_sz) / 2;
    if (nb + two_sz > ctx->norb) return fail(ctx, MBE_EINVAL, "alpha electrons exceed the orbitals");
    ctx->two_sz = two_sz;
    ctx->nocc = nb;
    ctx->nocc_a = nb + two_sz;
    ctx->have_ref = false;
    ctx->kept.clear();
    ctx->kept_ref = false;
    ctx->rdm_blocks.clear();
    ctx->guess_prev.clear();
    ctx->guess_cur.clear();
    ctx->last_order = 0;
    ctx->cur_order = 0;
    ctx->order_sums.clear();
    return MBE_OK;
  });
}

int mbe_set_reference(mbe_ctx* ctx, const int* ref_orbs, int nref, const int* exp_orbs, int nexp,
                      double* e_ref) {
  return guarded(ctx, [&]() -> int {
    if (ctx->norb == 0) return fail(ctx, MBE_ESTATE, "no integrals loaded");
    if (nref < 0 || nexp < 0 || (nref && !ref_orbs) || (nexp && !exp_orbs))
      return fail(ctx, MBE_EINVAL, "bad reference/expansion arguments");
    std::set<int> seen;
    for (int i = 0; i < nref; i++) {
      int o = ref_orbs[i];
      if (o < 0 || o >= ctx->norb || !seen.insert(o).second)
        return fail(ctx, MBE_EINVAL, "bad reference orbital");
    }
    // a high-spin reference determinant: its singly occupied orbitals belong
    // to the reference space (the inactive core stays closed-shell)
    for (int o = ctx->nocc; o < ctx->nocc_a; o++)
      if (!seen.count(o))
        return fail(ctx, MBE_EINVAL, "singly occupied orbitals must be in the reference space");
    for (int i = 0; i < nexp; i++) {
      int o = exp_orbs[i];
      if (o < 0 || o >= ctx->norb || !seen.insert(o).second)
        return fail(ctx, MBE_EINVAL, "bad or duplicate expansion orbital");
    }
    ctx->ref.assign(ref_orbs, ref_orbs + nref);
    std::sort(ctx->ref.begin(), ctx->ref.end());
    ctx->exp.assign(exp_orbs, exp_orbs + nexp);
    std::sort(ctx->exp.begin(), ctx->exp.end());
    // order 0: the CASCI of the reference space (a fresh warm-start chain)
    ctx->guess_prev.clear();
    ctx->guess_cur.clear();
    double e = 0.0;
    int32_t st = 0;
    std::vector<const double*> rdm;
    ctx->kept.clear();
    ctx->kept_ref = false;
    ctx->rdm_blocks.clear();
    if (nref > 0) {
      solve_jobs(ctx, {ctx->ref}, &e, &st, ctx->opt.keep_ci ? &rdm : nullptr, 0);
    } else {
      // empty reference: the inactive-core energy of the closed-shell determinant
      double ec = 0.0;
      const int n = ctx->norb;
      const int64_t NP = ctx->npair_g;
      auto gp = [](int p, int q) -> int64_t {
        return p >= q ? (int64_t)p * (p + 1) / 2 + q : (int64_t)q * (q + 1) / 2 + p;
      };
      for (int i = 0; i < ctx->nocc; i++) ec += 2.0 * ctx->h_host[(int64_t)i * n + i];
      for (int i = 0; i < ctx->nocc; i++)
        for (int j = 0; j < ctx->nocc; j++)
          ec += 2.0 * ctx->eri_host[gp(i, i) * NP + gp(j, j)] -
                ctx->eri_host[gp(i, j) * NP + gp(j, i)];
      e = ec;
    }
    ctx->e_ref = e;
    ctx->have_ref = true;
    if (ctx->opt.keep_ci && nref > 0) {
      ctx->ref_ci.order = 0;
      ctx->ref_ci.tuple.clear();
      ctx->ref_ci.n = nref;
      ctx->ref_ci.nsig = count_sig(ctx, ctx->ref);
      ctx->ref_ci.rdm = rdm[0];
      ctx->kept_ref = true;
    }
    hash_init(ctx, 4096);
    ctx->history.clear();
    ctx->last_order = 0;
    ctx->cur_order = 0;
    ctx->order_sums.clear();
    ctx->prev_tuples.clear();
    ctx->prev_keep.clear();
    ctx->prev_order = 0;
    ctx->pruned = false;
    ctx->partner.assign(ctx->norb, -1);
    if (e_ref) *e_ref = e;
    if (st != MBE_OK) return fail(ctx, MBE_ENOCONV, "reference CASCI did not converge");
    return MBE_OK;
  });
}

int mbe_solve_tuples(mbe_ctx* ctx, int order, const int32_t* tuples, int64_t ntup, double* e_out,
                     int32_t* status_out) {
  return guarded(ctx, [&]() -> int {
    if (!ctx->have_ref) return fail(ctx, MBE_ESTATE, "no reference space set");
    if (order < 1 || order > MBE_MAX_ORDER || ntup < 0 || (ntup && !tuples))
      return fail(ctx, MBE_EINVAL, "bad order or tuple arguments");
    std::set<int> expset(ctx->exp.begin(), ctx->exp.end());
    std::vector<std::vector<int>> acts(ntup);
    for (int64_t t = 0; t < ntup; t++) {
      const int32_t* row = tuples + t * order;
      for (int i = 0; i < order; i++) {
        if (!expset.count(row[i])) return fail(ctx, MBE_EINVAL, "tuple orbital not in expansion space");
        if (i && row[i] <= row[i - 1]) return fail(ctx, MBE_EINVAL, "tuple rows must be strictly ascending");
      }
      acts[t] = active_of(ctx, row, order);
    }
    std::vector<double> eps(ntup);
    std::vector<int32_t> st(ntup, 0);
    std::vector<const double*> rdm;
    if (ctx->opt.keep_ci) {
      // a re-solve of this order replaces the RDMs kept for it and above
      ctx->kept.erase(std::remove_if(ctx->kept.begin(), ctx->kept.end(),
                                     [&](const KeptRdm& k) { return k.order >= order; }),
                      ctx->kept.end());
      ctx->rdm_blocks.erase(std::remove_if(ctx->rdm_blocks.begin(), ctx->rdm_blocks.end(),
                                           [&](const RdmBlock& b) { return b.order >= order; }),
                            ctx->rdm_blocks.end());
    }
    solve_jobs(ctx, acts, eps.data(), st.data(), ctx->opt.keep_ci ? &rdm : nullptr, order);
    ctx->cur_order = order;
    ctx->cur_tuples.assign(tuples, tuples + ntup * order);
    ctx->cur_eps = eps;
    ctx->cur_tuples_dev.reset(&ctx->pool, (size_t)ntup * order);
    ctx->cur_eps_dev.reset(&ctx->pool, ntup);
    if (ntup) {
      CU_CHECK(cudaMemcpyAsync(ctx->cur_tuples_dev.ptr, tuples, sizeof(int32_t) * ntup * order,
                               cudaMemcpyHostToDevice, ctx->stream));
      CU_CHECK(cudaMemcpyAsync(ctx->cur_eps_dev.ptr, eps.data(), sizeof(double) * ntup,
                               cudaMemcpyHostToDevice, ctx->stream));
      CU_CHECK(cudaStreamSynchronize(ctx->stream));
    }
    if (ctx->opt.keep_ci) {
      for (int64_t t = 0; t < ntup; t++) {
        KeptRdm k;
        k.order = order;
        k.tuple.assign(tuples + t * order, tuples + (t + 1) * order);
        k.n = (int)acts[t].size();
        k.nsig = count_sig(ctx, acts[t]);
        k.rdm = rdm[t];
        ctx->kept.push_back(std::move(k));
      }
    }
    bool bad = false;
    for (int64_t t = 0; t < ntup; t++) {
      if (e_out) e_out[t] = eps[t];
      if (status_out) status_out[t] = st[t];
      bad |= st[t] != 0;
    }
    if (bad) return fail(ctx, MBE_ENOCONV, "some CASCI did not converge");
    return MBE_OK;
  });
}

int mbe_increments(mbe_ctx* ctx, int order, double screen_thr, double* inc_out, uint8_t* keep_out,
                   double* e_order_out, double* e_total_out) {
  return guarded(ctx, [&]() -> int {
    if (!ctx->have_ref) return fail(ctx, MBE_ESTATE, "no reference space set");
    if (order != ctx->last_order + 1 || order != ctx->cur_order)
      return fail(ctx, MBE_ESTATE, "increments must be processed order by order after solving");
    if (!(screen_thr >= 0.0)) return fail(ctx, MBE_EINVAL, "negative screening threshold");
    const int64_t ntup = (int64_t)ctx->cur_eps.size();
    if (2 * (ctx->hash.count + ntup) > ctx->hash.cap) {
      // grow the table and re-insert every processed order
      hash_init(ctx, 4 * (ctx->hash.count + ntup));
      for (const OrderRec& r : ctx->history) {
        int64_t nt = (int64_t)r.inc.size();
        if (!nt) continue;
        DevBuf<int32_t> tb(&ctx->pool, r.tuples.size());
        DevBuf<double> vb(&ctx->pool, nt);
        DevBuf<uint8_t> kb(&ctx->pool, nt);
        CU_CHECK(cudaMemcpyAsync(tb.ptr, r.tuples.data(), sizeof(int32_t) * r.tuples.size(),
                                 cudaMemcpyHostToDevice, ctx->stream));
        CU_CHECK(cudaMemcpyAsync(vb.ptr, r.inc.data(), sizeof(double) * nt, cudaMemcpyHostToDevice,
                                 ctx->stream));
        CU_CHECK(cudaMemcpyAsync(kb.ptr, r.keep.data(), nt, cudaMemcpyHostToDevice, ctx->stream));
        hash_insert(ctx, tb.ptr, r.order, nt, vb.ptr, kb.ptr);
      }
    }
    DevBuf<double> inc(&ctx->pool, std::max<int64_t>(ntup, 1));
    DevBuf<uint8_t> keep(&ctx->pool, std::max<int64_t>(ntup, 1));
    DevBuf<int32_t> err(&ctx->pool, 1);
    CU_CHECK(cudaMemsetAsync(err.ptr, 0, sizeof(int32_t), ctx->stream));
    increments_kernel_launch(ctx, ctx->cur_tuples_dev.ptr, order, ntup, ctx->cur_eps_dev.ptr,
                             ctx->e_ref, screen_thr, inc.ptr, keep.ptr, err.ptr);
    int32_t e = 0;
    CU_CHECK(cudaMemcpyAsync(&e, err.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    CU_CHECK(cudaStreamSynchronize(ctx->stream));
    if (e) return fail(ctx, MBE_ELOOKUP, "a subtuple increment is missing from the hash");
    hash_insert(ctx, ctx->cur_tuples_dev.ptr, order, ntup, inc.ptr, keep.ptr);
    double es = kahan_sum_device(ctx, inc.ptr, ntup);
    ctx->order_sums.push_back(es);
    std::vector<uint8_t> kh(ntup);
    if (ntup) {
      if (inc_out)
        CU_CHECK(cudaMemcpyAsync(inc_out, inc.ptr, sizeof(double) * ntup, cudaMemcpyDeviceToHost,
                                 ctx->stream));
      CU_CHECK(cudaMemcpyAsync(kh.data(), keep.ptr, ntup, cudaMemcpyDeviceToHost, ctx->stream));
      CU_CHECK(cudaStreamSynchronize(ctx->stream));
    }
    if (keep_out) std::memcpy(keep_out, kh.data(), ntup);
    OrderRec rec;
    rec.order = order;
    rec.tuples = ctx->cur_tuples;
    rec.eps = ctx->cur_eps;
    rec.inc.resize(ntup);
    if (ntup)
      CU_CHECK(cudaMemcpy(rec.inc.data(), inc.ptr, sizeof(double) * ntup, cudaMemcpyDeviceToHost));
    rec.keep = kh;
    ctx->history.push_back(std::move(rec));
    // total: eps_Pi + Kahan sum of the order sums
    double s = ctx->e_ref, c = 0.0;
    for (double v : ctx->order_sums) {
      double y = v - c, t = s + y;
      c = (t - s) - y;
      s = t;
    }
    if (e_order_out) *e_order_out = es;
    if (e_total_out) *e_total_out = s;
    ctx->last_order = order;
    ctx->prev_order = order;
    ctx->prev_tuples = ctx->cur_tuples;
    ctx->prev_keep = kh;
    return MBE_OK;
  });
}

int mbe_set_pruning_pairs(mbe_ctx* ctx, const int32_t* pairs, int npairs) {
  return guarded(ctx, [&]() -> int {
    if (!ctx->have_ref) return fail(ctx, MBE_ESTATE, "no reference space set");
    if (ctx->last_order != 0 || ctx->cur_order != 0)
      return fail(ctx, MBE_ESTATE, "pruning pairs must be set before the first order");
    if (npairs < 0 || (npairs && !pairs)) return fail(ctx, MBE_EINVAL, "bad pair arguments");
    std::vector<int32_t> part(ctx->norb, -1);
    std::set<int> expset(ctx->exp.begin(), ctx->exp.end());
    for (int i = 0; i < npairs; i++) {
      const int a = pairs[2 * i], b = pairs[2 * i + 1];
      if (a == b || !expset.count(a) || !expset.count(b) || part[a] >= 0 || part[b] >= 0)
        return fail(ctx, MBE_EINVAL, "pairs must join two distinct expansion orbitals, each once");
      part[a] = b;
      part[b] = a;
    }
    ctx->partner = part;
    ctx->pruned = npairs > 0;
    ctx->partner_dev.reset(&ctx->pool, std::max(1, ctx->norb));
    CU_CHECK(cudaMemcpyAsync(ctx->partner_dev.ptr, part.data(), sizeof(int32_t) * ctx->norb,
                             cudaMemcpyHostToDevice, ctx->stream));
    CU_CHECK(cudaStreamSynchronize(ctx->stream));
    return MBE_OK;
  });
}

int mbe_next_tuples(mbe_ctx* ctx, int order, int32_t* tuples_out, int64_t cap, int64_t* ntup_out) {
  return guarded(ctx, [&]() -> int {
    if (!ctx->have_ref) return fail(ctx, MBE_ESTATE, "no reference space set");
    if (!ntup_out) return fail(ctx, MBE_EINVAL, "null ntup_out");
    if (ctx->pruned) {
      if (order < 1 || order > MBE_MAX_ORDER || order != ctx->last_order + 1)
        return fail(ctx, MBE_ESTATE, "next tuples need the increments of order-1");
      std::vector<int32_t> t = next_tuples_pruned(ctx, order);
      const int64_t n = (int64_t)t.size() / order;
      *ntup_out = n;
      if (tuples_out) {
        if (cap < n) return fail(ctx, MBE_EINVAL, "output capacity too small");
        std::copy(t.begin(), t.end(), tuples_out);
      }
      return MBE_OK;
    }
    if (order == 1) {
      int64_t n = (int64_t)ctx->exp.size();
      *ntup_out = n;
      if (tuples_out) {
        if (cap < n) return fail(ctx, MBE_EINVAL, "output capacity too small");
        for (int64_t i = 0; i < n; i++) tuples_out[i] = ctx->exp[i];
      }
      return MBE_OK;
    }
    if (order < 2 || order > MBE_MAX_ORDER || order != ctx->last_order + 1)
      return fail(ctx, MBE_ESTATE, "next tuples need the increments of order-1");
    const int kp = order - 1;
    const int64_t np = (int64_t)ctx->prev_tuples.size() / kp;
    DevBuf<int32_t> par(&ctx->pool, std::max<int64_t>(1, np * kp));
    DevBuf<int32_t> ex(&ctx->pool, std::max<size_t>(1, ctx->exp.size()));
    if (np)
      CU_CHECK(cudaMemcpyAsync(par.ptr, ctx->prev_tuples.data(), sizeof(int32_t) * np * kp,
                               cudaMemcpyHostToDevice, ctx->stream));
    std::vector<int32_t> exh(ctx->exp.begin(), ctx->exp.end());
    if (!exh.empty())
      CU_CHECK(cudaMemcpyAsync(ex.ptr, exh.data(), sizeof(int32_t) * exh.size(),
                               cudaMemcpyHostToDevice, ctx->stream));
    DevBuf<int32_t> out;
    int64_t n = next_tuples_device(ctx, par.ptr, kp, np, ex.ptr, (int)exh.size(), out);
    *ntup_out = n;
    if (tuples_out) {
      if (cap < n) return fail(ctx, MBE_EINVAL, "output capacity too small");
      if (n)
        CU_CHECK(cudaMemcpyAsync(tuples_out, out.ptr, sizeof(int32_t) * n * order,
                                 cudaMemcpyDeviceToHost, ctx->stream));
      CU_CHECK(cudaStreamSynchronize(ctx->stream));
    }
    return MBE_OK;
  });
}

int mbe_energy_backward(mbe_ctx* ctx, double scale, double* dh, double* deri) {
  return guarded(ctx, [&]() -> int {
    if (!dh || !deri) return fail(ctx, MBE_EINVAL, "null output pointer");
    if (!ctx->norb) return fail(ctx, MBE_ESTATE, "no integrals loaded");
    if (ctx->opt.backward_share < 0 || ctx->opt.backward_share > 2)
      return fail(ctx, MBE_EINVAL, "backward_share must be 0, 1 or 2");
    return backward_run(ctx, scale, dh, deri);
  });
}

int mbe_get_stats(const mbe_ctx* ctx, mbe_stats* out) {
  if (!ctx || !out) return MBE_EINVAL;
  mbe_ctx* c = const_cast<mbe_ctx*>(ctx);
  cudaSetDevice(c->device);
  c->dom_timer.resolve();
  c->fp64_timer.resolve();
  *out = ctx->stats;
  out->launches = __atomic_load_n(&g_mbe_launches, __ATOMIC_RELAXED) - ctx->launch_base;
  out->host_launches =
      __atomic_load_n(&g_mbe_host_launches, __ATOMIC_RELAXED) - ctx->host_launch_base;
  out->dom_ms = c->dom_timer.ms;
  out->fp64_ms = c->fp64_timer.ms;
  return MBE_OK;
}

int mbe_reset_stats(mbe_ctx* ctx) {
  if (!ctx) return MBE_EINVAL;
  cudaSetDevice(ctx->device);
  ctx->dom_timer.resolve();
  ctx->dom_timer.ms = 0.0;
  ctx->fp64_timer.resolve();
  ctx->fp64_timer.ms = 0.0;
  ctx->stats = mbe_stats{};
  ctx->launch_base = __atomic_load_n(&g_mbe_launches, __ATOMIC_RELAXED);
  ctx->host_launch_base = __atomic_load_n(&g_mbe_host_launches, __ATOMIC_RELAXED);
  return MBE_OK;
}

int mbe_set_order_energies(mbe_ctx* ctx, int order, const int32_t* tuples, int64_t ntup,
                           const double* eps) {
  return guarded(ctx, [&]() -> int {
    if (!ctx->have_ref) return fail(ctx, MBE_ESTATE, "no reference space set");
    if (order < 1 || order > MBE_MAX_ORDER || ntup < 0 || (ntup && (!tuples || !eps)))
      return fail(ctx, MBE_EINVAL, "bad order or tuple arguments");
    std::set<int> expset(ctx->exp.begin(), ctx->exp.end());
    for (int64_t t = 0; t < ntup; t++) {
      const int32_t* row = tuples + t * order;
      if (!std::isfinite(eps[t])) return fail(ctx, MBE_EINVAL, "non-finite energy");
      for (int i = 0; i < order; i++) {
        if (!expset.count(row[i])) return fail(ctx, MBE_EINVAL, "tuple orbital not in expansion space");
        if (i && row[i] <= row[i - 1]) return fail(ctx, MBE_EINVAL, "tuple rows must be strictly ascending");
      }
    }
    ctx->cur_order = order;
    ctx->cur_tuples.assign(tuples, tuples + ntup * order);
    ctx->cur_eps.assign(eps, eps + ntup);
    ctx->cur_tuples_dev.reset(&ctx->pool, (size_t)ntup * order);
    ctx->cur_eps_dev.reset(&ctx->pool, ntup);
    if (ntup) {
      CU_CHECK(cudaMemcpyAsync(ctx->cur_tuples_dev.ptr, tuples, sizeof(int32_t) * ntup * order,
                               cudaMemcpyHostToDevice, ctx->stream));
      CU_CHECK(cudaMemcpyAsync(ctx->cur_eps_dev.ptr, eps, sizeof(double) * ntup,
                               cudaMemcpyHostToDevice, ctx->stream));
      CU_CHECK(cudaStreamSynchronize(ctx->stream));
    }
    return MBE_OK;
  });
}

int mbe_sigma_noalloc(mbe_ctx* ctx, const int* act, int nact, const double* c_dev,
                      double* sigma_dev, int64_t ndet, double* e_core) {
  return guarded(ctx, [&]() -> int {
    return noalloc_sigma_run(ctx, act, nact, c_dev, sigma_dev, ndet, e_core);
  });
}

int mbe_sigma(mbe_ctx* ctx, const int* act, int nact, const double* c, double* sigma,
              double* e_core) {
  return guarded(ctx, [&]() -> int {
    if (ctx->norb == 0) return fail(ctx, MBE_ESTATE, "no integrals loaded");
    if (nact < 1 || nact > 15 || !act || !c || !sigma)
      return fail(ctx, MBE_EINVAL, "bad sigma arguments");
    std::vector<int> a(act, act + nact);
    std::sort(a.begin(), a.end());
    for (int i = 0; i < nact; i++)
      if (a[i] < 0 || a[i] >= ctx->norb || (i && a[i] == a[i - 1]))
        return fail(ctx, MBE_EINVAL, "bad active orbital");
    for (int o = ctx->nocc; o < ctx->nocc_a; o++)
      if (!std::binary_search(a.begin(), a.end(), o))
        return fail(ctx, MBE_EINVAL, "singly occupied orbitals must be active");
    const int nsig = count_sig(ctx, a), nsigb = count_sig_b(ctx, a);
    StringTables* tab = get_tables(ctx, nact, nsig);
    StringTables* tabb = nsigb == nsig ? tab : get_tables(ctx, nact, nsigb);
    BinProblem bp;
    bp.n = nact;
    bp.nsig = nsig;
    bp.nstr = tab->nstr;
    bp.npair = tab->npair;
    bp.nsigb = nsigb;
    bp.nstrb = tabb->nstr;
    bp.ndet = (int64_t)tab->nstr * tabb->nstr;
    bp.B = 1;
    bp.tab = tab;
    bp.tabb = tabb;
    bp.act.reset(&ctx->pool, nact);
    std::vector<int32_t> a32(a.begin(), a.end());
    CU_CHECK(cudaMemcpyAsync(bp.act.ptr, a32.data(), sizeof(int32_t) * nact, cudaMemcpyHostToDevice,
                             ctx->stream));
    launch_effints(ctx, bp);
    DevBuf<double> cd(&ctx->pool, bp.ndet), sd(&ctx->pool, bp.ndet);
    CU_CHECK(cudaMemcpyAsync(cd.ptr, c, sizeof(double) * bp.ndet, cudaMemcpyHostToDevice,
                             ctx->stream));
    SigmaWork w;
    // mixed precision: the tensor-core path (valid for c = c^T, the
    // alpha<->beta symmetric sector of a closed shell), else FP64
    if (ctx->opt.precision == MBE_MIXED_BF16X3 && bp.closed() && sigma_tc_supported(nact, bp.nstr)) {
      // the mixed mode keeps its vectors in FP32
      std::vector<float> cf(c, c + bp.ndet), sf(bp.ndet);
      DevBuf<float> cdf(&ctx->pool, bp.ndet), sdf(&ctx->pool, bp.ndet);
      CU_CHECK(cudaMemcpyAsync(cdf.ptr, cf.data(), sizeof(float) * bp.ndet, cudaMemcpyHostToDevice,
                               ctx->stream));
      sigma_tc(ctx, bp, w, cdf.ptr, bp.ndet, sdf.ptr, bp.ndet, nullptr, ctx->opt.spin_shift);
      if (sigma_tc_error(ctx, w)) return fail(ctx, MBE_ETIMEOUT, "tensor-core sigma wait timed out");
      CU_CHECK(cudaMemcpyAsync(sf.data(), sdf.ptr, sizeof(float) * bp.ndet, cudaMemcpyDeviceToHost,
                               ctx->stream));
      double ec = 0.0;
      CU_CHECK(cudaMemcpyAsync(&ec, bp.ecore.ptr, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
      CU_CHECK(cudaStreamSynchronize(ctx->stream));
      for (int64_t i = 0; i < bp.ndet; i++) sigma[i] = sf[i];
      if (e_core) *e_core = ec;
      return MBE_OK;
    } else {
      // emulated FP64: the fused exact kernel for vectors like the mixed
      // mode's exact points (c = c^T with FP32 values, |c_i| <= 1), else the
      // sliced contraction on HBM intermediates
      bool fused = ctx->opt.precision == MBE_EMULATED_FP64 && bp.closed() &&
                   sigma_exact_supported(bp.npair, bp.nstr);
      for (int64_t i = 0; fused && i < bp.nstr; i++)
        for (int64_t j = 0; j <= i; j++) {
          const double x = c[i * bp.nstr + j];
          if (x != c[j * bp.nstr + i] || (double)(float)x != x || std::fabs(x) > 1.0) {
            fused = false;
            break;
          }
        }
      if (fused) {
        std::vector<float> cf(c, c + bp.ndet);
        DevBuf<float> cdf(&ctx->pool, bp.ndet);
        CU_CHECK(cudaMemcpyAsync(cdf.ptr, cf.data(), sizeof(float) * bp.ndet, cudaMemcpyHostToDevice,
                                 ctx->stream));
        sigma_exact(ctx, bp, w, cdf.ptr, bp.ndet, sd.ptr, bp.ndet, nullptr);
        launch_finish_sym_fp64(ctx, bp, sd.ptr, bp.ndet, cd.ptr, bp.ndet, ctx->opt.spin_shift,
                               nullptr);
        if (sigma_tc_error(ctx, w)) return fail(ctx, MBE_ETIMEOUT, "fused exact sigma wait timed out");
      } else {
        const bool emu = ctx->opt.precision == MBE_EMULATED_FP64 && ozaki_supported(bp.npair);
        sigma_fp64(ctx, bp, w, cd.ptr, bp.ndet, sd.ptr, bp.ndet, nullptr, ctx->opt.spin_shift, emu);
        if (emu && sigma_tc_error(ctx, w))
          return fail(ctx, MBE_ETIMEOUT, "tensor-core contraction wait timed out");
      }
    }
    CU_CHECK(cudaMemcpyAsync(sigma, sd.ptr, sizeof(double) * bp.ndet, cudaMemcpyDeviceToHost,
                             ctx->stream));
    double ec = 0.0;
    CU_CHECK(cudaMemcpyAsync(&ec, bp.ecore.ptr, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CU_CHECK(cudaStreamSynchronize(ctx->stream));
    if (e_core) *e_core = ec;
    return MBE_OK;
  });
}

}  // extern "C"
