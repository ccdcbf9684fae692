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

// Eq. 3: inc_T = eps_T - eps_Pi - sum over proper non-empty subtuples S of
// inc_S (all looked up in the hash).  Compensated summation, subsets visited
// in increasing bit-mask order.
__global__ void k_increments(DevHash h, const int32_t* __restrict__ tuples, int order, int64_t ntup,
                             const double* __restrict__ eps, double eps_ref, double thr,
                             double* __restrict__ inc, uint8_t* __restrict__ keep_out,
                             int32_t* err) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntup) return;
  int orb[MBE_MAX_ORDER];
  for (int i = 0; i < order; i++) orb[i] = tuples[t * order + i];
  double s = eps[t] - eps_ref, comp = 0.0;
  const unsigned full = (1u << order) - 1u;
  for (unsigned m = 1; m < full; m++) {
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
__global__ void k_mbe_coef(DevHash h, const int32_t* __restrict__ tuples, int order, int64_t ntup,
                           int32_t* __restrict__ coef, int32_t* __restrict__ coef_ref,
                           int32_t* __restrict__ err) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntup) return;
  int orb[MBE_MAX_ORDER];
  for (int i = 0; i < order; i++) orb[i] = tuples[t * order + i];
  const unsigned full = (1u << order) - 1u;
  for (unsigned m = 1; m <= full; m++) {
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
    atomicAdd(&coef[slot], ((order - __popc(m)) & 1) ? -1 : 1);
  }
  atomicAdd(coef_ref, (order & 1) ? -1 : 1);
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
      dev_hash(ctx), tuples_dev, order, ntup, eps_dev, eps_ref, thr, inc_dev, keep_dev, err_dev);
  CU_LAUNCH_CHECK();
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
      dev_hash(ctx), tuples_dev, order, ntup, coef_dev, coef_ref_dev, err_dev);
  CU_LAUNCH_CHECK();
}
