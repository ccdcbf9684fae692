// Increment assembly of Eq. 3 by tuple-hash lookup (K9), compensated order
// sums (K10) and next-order tuple generation with screening (a1).
//
// A tuple is keyed by its 128-bit orbital set.  The hash is open addressing
// with linear probing; a slot is claimed with atomicCAS on its state word.
// Inserts of one order run in their own launch after every lookup of that
// order has finished, so lookups never race with inserts.
#include "mbe_internal.cuh"
#include <algorithm>

namespace {

__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

__device__ __forceinline__ unsigned long long hkey(unsigned long long k0, unsigned long long k1) {
  return mix64(k0 ^ mix64(k1 + 0x632be59bd9b4e019ull));
}

struct DevHash {
  const unsigned long long* keys;
  const double* val;
  const uint8_t* keep;
  const int32_t* state;
  int64_t mask;
};

// returns slot index or -1
__device__ int64_t hash_find(const DevHash& h, unsigned long long k0, unsigned long long k1) {
  int64_t s = (int64_t)(hkey(k0, k1) & (unsigned long long)h.mask);
  for (int64_t probe = 0; probe <= h.mask; probe++) {
    if (h.state[s] == 0) return -1;
    if (h.keys[2 * s] == k0 && h.keys[2 * s + 1] == k1) return s;
    s = (s + 1) & h.mask;
  }
  return -1;
}

__global__ void k_hash_insert(unsigned long long* keys, double* val, uint8_t* keep, int32_t* state,
                              int64_t mask, const int32_t* __restrict__ tuples, int order,
                              int64_t ntup, const double* __restrict__ vals,
                              const uint8_t* __restrict__ keeps, int32_t* err) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntup) return;
  unsigned long long k0 = 0, k1 = 0;
  for (int i = 0; i < order; i++) {
    int o = tuples[t * order + i];
    if (o < 64) k0 |= 1ull << o; else k1 |= 1ull << (o - 64);
  }
  int64_t s = (int64_t)(hkey(k0, k1) & (unsigned long long)mask);
  for (int64_t probe = 0; probe <= mask; probe++) {
    if (atomicCAS(&state[s], 0, 1) == 0) {
      keys[2 * s] = k0;
      keys[2 * s + 1] = k1;
      val[s] = vals[t];
      keep[s] = keeps ? keeps[t] : 1;
      return;
    }
    s = (s + 1) & mask;
  }
  atomicExch(err, MBE_ENOMEM);
}

// pi-pruning: for position i of a tuple, the bit of its partner's position
// (0 for an orbital without partner); a subset m of the positions is a union
// of units iff it holds the partner of each of its members
__device__ __forceinline__ void partner_bits(const int* orb, int order,
                                             const int32_t* __restrict__ partner, unsigned* pb) {
  for (int i = 0; i < order; i++) {
    pb[i] = 0u;
    if (!partner) continue;
    const int p = partner[orb[i]];
    for (int j = 0; j < order; j++)
      if (orb[j] == p) pb[i] = 1u << j;
  }
}
__device__ __forceinline__ bool unit_closed(unsigned m, const unsigned* pb, int order) {
  unsigned need = 0u;
  for (int i = 0; i < order; i++)
    if ((m >> i) & 1u) need |= pb[i];
  return (need & ~m) == 0u;
}
// number of units in a unit-closed subset: each pair counted once
__device__ __forceinline__ int unit_count(unsigned m, const unsigned* pb, int order) {
  int n = 0;
  for (int i = 0; i < order; i++)
    if (((m >> i) & 1u) && (pb[i] == 0u || pb[i] > (1u << i))) n++;
  return n;
}

// Eq. 3: inc_T = eps_T - eps_Pi - sum over proper non-empty subtuples S of
// inc_S (all looked up in the hash); with pi-pruning (partner != NULL) over
// the proper non-empty unions of units.  Compensated summation, subsets
// visited in increasing bit-mask order.
__global__ void k_increments(DevHash h, const int32_t* __restrict__ tuples, int order, int64_t ntup,
                             const double* __restrict__ eps, double eps_ref, double thr,
                             const int32_t* __restrict__ partner, double* __restrict__ inc,
                             uint8_t* __restrict__ keep_out, int32_t* err) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntup) return;
  int orb[MBE_MAX_ORDER];
  unsigned pb[MBE_MAX_ORDER];
  for (int i = 0; i < order; i++) orb[i] = tuples[t * order + i];
  partner_bits(orb, order, partner, pb);
  double s = eps[t] - eps_ref, comp = 0.0;
  const unsigned full = (1u << order) - 1u;
  for (unsigned m = 1; m < full; m++) {
    if (partner && !unit_closed(m, pb, order)) continue;
    unsigned long long k0 = 0, k1 = 0;
    for (int i = 0; i < order; i++)
      if ((m >> i) & 1u) {
        int o = orb[i];
        if (o < 64) k0 |= 1ull << o; else k1 |= 1ull << (o - 64);
      }
    int64_t slot = hash_find(h, k0, k1);
    if (slot < 0) {
      atomicExch(err, MBE_ELOOKUP);
      continue;
    }
    double y = -h.val[slot] - comp;
    double tt = s + y;
    comp = (tt - s) - y;
    s = tt;
  }
  inc[t] = s;
  keep_out[t] = (fabs(s) >= thr) ? 1 : 0;
}

// Kahan sum of v[0..n) by one block: per-thread compensated partial sums in
// a fixed stride, then a fixed-order compensated combination.
__global__ void k_kahan(const double* __restrict__ v, int64_t n, double* out) {
  __shared__ double ss[1024], sc[1024];
  double s = 0.0, c = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    double y = v[i] - c;
    double t = s + y;
    c = (t - s) - y;
    s = t;
  }
  ss[threadIdx.x] = s;
  sc[threadIdx.x] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    double S = 0.0, C = 0.0;
    for (int i = 0; i < (int)blockDim.x; i++) {
      double y = (ss[i] - sc[i]) - C;
      double t = S + y;
      C = (t - S) - y;
      S = t;
    }
    *out = S;
  }
}

// Candidate (parent p, expansion orbital e): T = parent + exp[e] if exp[e]
// exceeds the parent's last orbital; kept iff all order-1 subtuples exist
// and at least one is kept.
__device__ bool candidate_ok(const DevHash& h, const int32_t* parents, int kp, int64_t p,
                             const int32_t* exp, int e, int* orb) {
  const int32_t* par = parents + p * kp;
  int o = exp[e];
  if (kp > 0 && o <= par[kp - 1]) return false;
  for (int i = 0; i < kp; i++) orb[i] = par[i];
  orb[kp] = o;
  const int k = kp + 1;
  bool any_keep = false;
  for (int drop = 0; drop < k; drop++) {
    unsigned long long k0 = 0, k1 = 0;
    for (int i = 0; i < k; i++) {
      if (i == drop) continue;
      int x = orb[i];
      if (x < 64) k0 |= 1ull << x; else k1 |= 1ull << (x - 64);
    }
    int64_t slot = hash_find(h, k0, k1);
    if (slot < 0) return false;
    if (h.keep[slot]) any_keep = true;
  }
  return any_keep;
}

constexpr int GEN_BLOCK = 256;

__global__ void k_gen_count(DevHash h, const int32_t* __restrict__ parents, int kp, int64_t np,
                            const int32_t* __restrict__ exp, int nexp, int32_t* __restrict__ bcount) {
  int64_t c = (int64_t)blockIdx.x * GEN_BLOCK + threadIdx.x;
  int ok = 0;
  int orb[MBE_MAX_ORDER + 1];
  if (c < np * nexp) ok = candidate_ok(h, parents, kp, c / nexp, exp, (int)(c % nexp), orb);
  int cnt = __syncthreads_count(ok);
  if (threadIdx.x == 0) bcount[blockIdx.x] = cnt;
}

// exclusive scan of block counts (one block, serial chunks per thread)
__global__ void k_scan(const int32_t* __restrict__ cnt, int64_t nb, int64_t* __restrict__ off,
                       int64_t* __restrict__ total) {
  __shared__ int64_t part[1024];
  int64_t per = (nb + blockDim.x - 1) / blockDim.x;
  int64_t a = threadIdx.x * per, b = min(nb, a + per);
  int64_t s = 0;
  for (int64_t i = a; i < b; i++) s += cnt[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t run = 0;
    for (int i = 0; i < (int)blockDim.x; i++) {
      int64_t v = part[i];
      part[i] = run;
      run += v;
    }
    *total = run;
  }
  __syncthreads();
  s = part[threadIdx.x];
  for (int64_t i = a; i < b; i++) {
    off[i] = s;
    s += cnt[i];
  }
}

__global__ void k_gen_write(DevHash h, const int32_t* __restrict__ parents, int kp, int64_t np,
                            const int32_t* __restrict__ exp, int nexp,
                            const int64_t* __restrict__ off, int32_t* __restrict__ out) {
  int64_t c = (int64_t)blockIdx.x * GEN_BLOCK + threadIdx.x;
  int orb[MBE_MAX_ORDER + 1];
  int ok = 0;
  if (c < np * nexp) ok = candidate_ok(h, parents, kp, c / nexp, exp, (int)(c % nexp), orb);
  __shared__ int wsum[GEN_BLOCK / 32];
  unsigned bal = __ballot_sync(0xffffffffu, ok);
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) wsum[warp] = __popc(bal);
  __syncthreads();
  int before = 0;
  for (int w = 0; w < warp; w++) before += wsum[w];
  before += __popc(bal & ((1u << lane) - 1u));
  if (ok) {
    int64_t pos = off[blockIdx.x] + before;
    for (int i = 0; i <= kp; i++) out[pos * (kp + 1) + i] = orb[i];
  }
}


// MBE coefficient of every processed tuple (Moebius inversion of Eq. 3):
// each tuple T adds (-1)^(|T| - |S|) to the coefficient of every non-empty
// subtuple S (itself included); the empty subtuple is counted in coef_ref.
// With pi-pruning (partner != NULL) the subtuples are the unions of units
// and the sign counts units.
__global__ void k_mbe_coef(DevHash h, const int32_t* __restrict__ tuples, int order, int64_t ntup,
                           const int32_t* __restrict__ partner, int32_t* __restrict__ coef,
                           int32_t* __restrict__ coef_ref, int32_t* __restrict__ err) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntup) return;
  int orb[MBE_MAX_ORDER];
  unsigned pb[MBE_MAX_ORDER];
  for (int i = 0; i < order; i++) orb[i] = tuples[t * order + i];
  partner_bits(orb, order, partner, pb);
  const unsigned full = (1u << order) - 1u;
  const int nt = partner ? unit_count(full, pb, order) : order;
  for (unsigned m = 1; m <= full; m++) {
    if (partner && !unit_closed(m, pb, order)) continue;
    unsigned long long k0 = 0, k1 = 0;
    for (int i = 0; i < order; i++)
      if ((m >> i) & 1u) {
        const int o = orb[i];
        if (o < 64) k0 |= 1ull << o; else k1 |= 1ull << (o - 64);
      }
    const int64_t slot = hash_find(h, k0, k1);
    if (slot < 0) {
      atomicExch(err, MBE_ELOOKUP);
      continue;
    }
    const int ns = partner ? unit_count(m, pb, order) : __popc(m);
    atomicAdd(&coef[slot], ((nt - ns) & 1) ? -1 : 1);
  }
  atomicAdd(coef_ref, (nt & 1) ? -1 : 1);
}

// pi-pruned generation: candidate (parent p of order kp, unit u) with the
// unit (ua, ub) (ub = -1 for a single orbital) added; formed iff the unit's
// lowest orbital exceeds the lowest orbital of every unit of the parent (each
// tuple has one canonical parent), every one-unit-removed subtuple exists
// (the empty one is the reference space) and, if any exists besides the
// empty one, at least one of them is kept.  Writes the tuple sorted.
__device__ bool candidate_ok_units(const DevHash& h, const int32_t* parents, int kp, int64_t p,
                                   const int32_t* ua, const int32_t* ub, int u,
                                   const int32_t* __restrict__ partner, int* orb) {
  const int32_t* par = parents + p * kp;
  const int a = ua[u], b = ub[u];
  for (int i = 0; i < kp; i++) {
    const int o = par[i], q = partner[o];
    const int lo = q >= 0 && q < o ? q : o;        // lowest orbital of o's unit
    if (lo >= a) return false;
  }
  const int k = kp + (b >= 0 ? 2 : 1);
  int n = 0, ia = 0;
  // merge the unit's orbitals into the sorted parent
  for (int i = 0; i < kp; i++) {
    while (ia < 2 && (ia == 0 ? a : b) >= 0 && (ia == 0 ? a : b) < par[i]) orb[n++] = ia++ == 0 ? a : b;
    orb[n++] = par[i];
  }
  while (ia < 2 && (ia == 0 ? a : b) >= 0) orb[n++] = ia++ == 0 ? a : b;
  if (n != k) return false;
  unsigned pb[MBE_MAX_ORDER + 2];
  partner_bits(orb, k, partner, pb);
  bool any_keep = false, any = false;
  for (int drop = 0; drop < k; drop++) {
    // remove the unit of position drop (once per unit: from its first member)
    if (pb[drop] && pb[drop] < (1u << drop)) continue;
    const unsigned rm = (1u << drop) | pb[drop];
    unsigned long long k0 = 0, k1 = 0;
    int cnt = 0;
    for (int i = 0; i < k; i++) {
      if ((rm >> i) & 1u) continue;
      const int x = orb[i];
      if (x < 64) k0 |= 1ull << x; else k1 |= 1ull << (x - 64);
      cnt++;
    }
    if (cnt == 0) continue;                        // the reference space
    any = true;
    const int64_t slot = hash_find(h, k0, k1);
    if (slot < 0) return false;
    if (h.keep[slot]) any_keep = true;
  }
  return any ? any_keep : true;
}

__global__ void k_gen_units(DevHash h, const int32_t* __restrict__ parents, int kp, int64_t np,
                            const int32_t* __restrict__ ua, const int32_t* __restrict__ ub, int nu,
                            const int32_t* __restrict__ partner, int k,
                            int32_t* __restrict__ count, int32_t* __restrict__ out, int64_t cap) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= np * nu) return;
  int orb[MBE_MAX_ORDER + 2];
  if (!candidate_ok_units(h, parents, kp, c / nu, ua, ub, (int)(c % nu), partner, orb)) return;
  const int pos = atomicAdd(count, 1);
  if (pos < cap)
    for (int i = 0; i < k; i++) out[(int64_t)pos * k + i] = orb[i];
}

DevHash dev_hash(mbe_ctx* ctx) {
  DevHash h;
  h.keys = ctx->hash.keys.ptr;
  h.val = ctx->hash.val.ptr;
  h.keep = ctx->hash.keep.ptr;
  h.state = ctx->hash.state.ptr;
  h.mask = ctx->hash.cap - 1;
  return h;
}

}  // namespace

void hash_init(mbe_ctx* ctx, int64_t cap) {
  int64_t c = 1024;
  while (c < cap) c <<= 1;
  HashTable& H = ctx->hash;
  H.cap = c;
  H.count = 0;
  H.keys.reset(&ctx->pool, 2 * c);
  H.val.reset(&ctx->pool, c);
  H.keep.reset(&ctx->pool, c);
  H.state.reset(&ctx->pool, c);
  CU_CHECK(cudaMemsetAsync(H.state.ptr, 0, sizeof(int32_t) * c, ctx->stream));
}

void hash_insert(mbe_ctx* ctx, const int32_t* tuples_dev, int order, int64_t ntup,
                 const double* vals_dev, const uint8_t* keep_dev) {
  if (ntup == 0) return;
  HashTable& H = ctx->hash;
  DevBuf<int32_t> err(&ctx->pool, 1);
  CU_CHECK(cudaMemsetAsync(err.ptr, 0, sizeof(int32_t), ctx->stream));
  k_hash_insert<<<(unsigned)((ntup + 255) / 256), 256, 0, ctx->stream>>>(
      H.keys.ptr, H.val.ptr, H.keep.ptr, H.state.ptr, H.cap - 1, tuples_dev, order, ntup,
      vals_dev, keep_dev, err.ptr);
  CU_LAUNCH_CHECK();
  int32_t e = 0;
  CU_CHECK(cudaMemcpyAsync(&e, err.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  CU_CHECK(cudaStreamSynchronize(ctx->stream));
  if (e) throw MbeError{MBE_ENOMEM, "tuple hash is full"};
  H.count += ntup;
}

void increments_kernel_launch(mbe_ctx* ctx, const int32_t* tuples_dev, int order, int64_t ntup,
                              const double* eps_dev, double eps_ref, double thr, double* inc_dev,
                              uint8_t* keep_dev, int32_t* err_dev) {
  if (ntup == 0) return;
  k_increments<<<(unsigned)((ntup + 127) / 128), 128, 0, ctx->stream>>>(
      dev_hash(ctx), tuples_dev, order, ntup, eps_dev, eps_ref, thr,
      ctx->pruned ? ctx->partner_dev.ptr : nullptr, inc_dev, keep_dev, err_dev);
  CU_LAUNCH_CHECK();
}

// pi-pruned tuples of order k: single units added to the order-(k-1) tuples
// and pair units added to the order-(k-2) tuples (for k = 2 the empty tuple),
// in lexicographic order
std::vector<int32_t> next_tuples_pruned(mbe_ctx* ctx, int k) {
  std::vector<int32_t> sa, sb, pa, pbv;
  for (int o : ctx->exp) {
    const int q = ctx->partner[o];
    if (q < 0) {
      sa.push_back(o);
      sb.push_back(-1);
    } else if (o < q) {
      pa.push_back(o);
      pbv.push_back(q);
    }
  }
  auto level = [&](int order) -> std::vector<int32_t> {
    for (const OrderRec& r : ctx->history)
      if (r.order == order) return r.tuples;
    return {};
  };
  std::vector<std::vector<int32_t>> found;
  DevHash h = dev_hash(ctx);
  for (int pass = 0; pass < 2; pass++) {
    const int kp = k - (pass == 0 ? 1 : 2);
    const std::vector<int32_t>& ua = pass == 0 ? sa : pa;
    const std::vector<int32_t>& ub = pass == 0 ? sb : pbv;
    if (kp < 0 || ua.empty()) continue;
    std::vector<int32_t> par = kp == 0 ? std::vector<int32_t>{} : level(kp);
    const int64_t np = kp == 0 ? 1 : (int64_t)par.size() / kp;
    if (np == 0) continue;
    const int nu = (int)ua.size();
    DevBuf<int32_t> dpar(&ctx->pool, std::max<size_t>(1, par.size())), dua(&ctx->pool, nu),
        dub(&ctx->pool, nu), cnt(&ctx->pool, 1);
    if (!par.empty())
      CU_CHECK(cudaMemcpyAsync(dpar.ptr, par.data(), sizeof(int32_t) * par.size(),
                               cudaMemcpyHostToDevice, ctx->stream));
    CU_CHECK(cudaMemcpyAsync(dua.ptr, ua.data(), sizeof(int32_t) * nu, cudaMemcpyHostToDevice,
                             ctx->stream));
    CU_CHECK(cudaMemcpyAsync(dub.ptr, ub.data(), sizeof(int32_t) * nu, cudaMemcpyHostToDevice,
                             ctx->stream));
    const int64_t cap = np * nu;
    DevBuf<int32_t> out(&ctx->pool, (size_t)cap * k);
    CU_CHECK(cudaMemsetAsync(cnt.ptr, 0, sizeof(int32_t), ctx->stream));
    k_gen_units<<<(unsigned)((cap + 255) / 256), 256, 0, ctx->stream>>>(
        h, dpar.ptr, kp, np, dua.ptr, dub.ptr, nu, ctx->partner_dev.ptr, k, cnt.ptr, out.ptr, cap);
    CU_LAUNCH_CHECK();
    int32_t n = 0;
    CU_CHECK(cudaMemcpyAsync(&n, cnt.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    CU_CHECK(cudaStreamSynchronize(ctx->stream));
    std::vector<int32_t> hv((size_t)n * k);
    if (n)
      CU_CHECK(cudaMemcpy(hv.data(), out.ptr, sizeof(int32_t) * hv.size(), cudaMemcpyDeviceToHost));
    for (int32_t i = 0; i < n; i++) found.emplace_back(hv.begin() + (size_t)i * k, hv.begin() + (size_t)(i + 1) * k);
  }
  std::sort(found.begin(), found.end());
  std::vector<int32_t> flat;
  flat.reserve(found.size() * k);
  for (const auto& t : found) flat.insert(flat.end(), t.begin(), t.end());
  return flat;
}

double kahan_sum_device(mbe_ctx* ctx, const double* v, int64_t n) {
  if (n == 0) return 0.0;
  DevBuf<double> out(&ctx->pool, 1);
  k_kahan<<<1, 1024, 0, ctx->stream>>>(v, n, out.ptr);
  CU_LAUNCH_CHECK();
  double r = 0.0;
  CU_CHECK(cudaMemcpyAsync(&r, out.ptr, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CU_CHECK(cudaStreamSynchronize(ctx->stream));
  return r;
}

int64_t next_tuples_device(mbe_ctx* ctx, const int32_t* parents_dev, int order_prev,
                           int64_t nparents, const int32_t* exp_dev, int nexp,
                           DevBuf<int32_t>& out) {
  int64_t ncand = nparents * (int64_t)nexp;
  if (ncand == 0) {
    out.reset(&ctx->pool, 0);
    return 0;
  }
  int64_t nb = (ncand + GEN_BLOCK - 1) / GEN_BLOCK;
  DevBuf<int32_t> cnt(&ctx->pool, nb);
  DevBuf<int64_t> off(&ctx->pool, nb), tot(&ctx->pool, 1);
  DevHash h = dev_hash(ctx);
  k_gen_count<<<(unsigned)nb, GEN_BLOCK, 0, ctx->stream>>>(h, parents_dev, order_prev, nparents,
                                                          exp_dev, nexp, cnt.ptr);
  CU_LAUNCH_CHECK();
  k_scan<<<1, 1024, 0, ctx->stream>>>(cnt.ptr, nb, off.ptr, tot.ptr);
  CU_LAUNCH_CHECK();
  int64_t total = 0;
  CU_CHECK(cudaMemcpyAsync(&total, tot.ptr, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
  CU_CHECK(cudaStreamSynchronize(ctx->stream));
  out.reset(&ctx->pool, (size_t)total * (order_prev + 1));
  if (total)
    k_gen_write<<<(unsigned)nb, GEN_BLOCK, 0, ctx->stream>>>(h, parents_dev, order_prev, nparents,
                                                            exp_dev, nexp, off.ptr, out.ptr);
  CU_LAUNCH_CHECK();
  return total;
}

void mbe_coef_launch(mbe_ctx* ctx, const int32_t* tuples_dev, int order, int64_t ntup,
                     int32_t* coef_dev, int32_t* coef_ref_dev, int32_t* err_dev) {
  if (ntup == 0) return;
  k_mbe_coef<<<(unsigned)((ntup + 127) / 128), 128, 0, ctx->stream>>>(
      dev_hash(ctx), tuples_dev, order, ntup, ctx->pruned ? ctx->partner_dev.ptr : nullptr,
      coef_dev, coef_ref_dev, err_dev);
  CU_LAUNCH_CHECK();
}
