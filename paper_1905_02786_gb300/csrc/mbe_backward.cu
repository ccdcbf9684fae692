// Energy gradient of the MBE energy with respect to the integrals (K11,
// K12).  E_MBE = eps_Pi + sum of the increments of Eq. 3 is linear in the
// tuple energies, E_MBE = sum_S c_S eps_S with
//   c_S = sum over tuples T of the set (and the empty tuple) with T >= S of
//         (-1)^(|T| - |S|)
// (the Moebius inversion of Eq. 3).  Every eps_S is stationary in its CI
// coefficients (Hellmann-Feynman), so
//   dE/dh_pq      = sum_S c_S gamma^S_pq
//   dE/d(pq|rs)   = 1/2 sum_S c_S Gamma^S_pqrs
// with the spin-summed full-space RDMs of each CASCI: inside the active
// space gamma^A and Gamma^A from the CI vector, with the closed-shell
// inactive core the factorised form Gamma_pqrs = gamma_pq gamma_rs
// - 1/2 gamma_ps gamma_rq (gamma = 2 on the core).
//   gamma+_P = c . D_P and Gamma'_PQ = D_P . D_Q with D_P = E+_P c give the
//   active RDMs in packed pairs: sum over the images of (pq), (rs) of
//   <E_pq E_rs> is Gamma'_PQ and Gamma_pqrs = <E_pq E_rs> - d_qr gamma_ps.
// The gradient w.r.t. the symmetric packed ERI matrix eri[P][Q] sums
// dE/d(pq|rs) over the full-tensor images of (P, Q) and is symmetrised.
//
// The RDMs are formed on the device as soon as a batch of CASCIs has
// converged (rdm_batch, called by the solver when keep_ci is set) and kept
// there, packed (gamma+ and the upper triangle of Gamma'); the backward then
// only weights and scatters them.  No CI vector is copied to the host.
#include "mbe_internal.cuh"
#include <algorithm>
#include <cmath>

namespace {

constexpr int RD_THREADS = 256, RD_BT = 32;

template <typename T>
__device__ __forceinline__ void load4(const T* p, T (&v)[4]);
template <>
__device__ __forceinline__ void load4<float>(const float* p, float (&v)[4]) {
  const float4 x = *reinterpret_cast<const float4*>(p);
  v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
}
template <>
__device__ __forceinline__ void load4<double>(const double* p, double (&v)[4]) {
  const double2 x = reinterpret_cast<const double2*>(p)[0];
  const double2 y = reinterpret_cast<const double2*>(p)[1];
  v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
}

// Partial sums of the Gram matrix of the rows D_0 .. D_{npair-1} and c over
// one chunk of determinants K = (a, b) of one vector (blockIdx.y):
//   D_P(a, b) = s c(J_a(P), b) + s' c(a, J_b(P))     (E+_P acting on c)
// (alpha links of a from `link`, beta links of b from `linkb`; c is
// nstr_alpha x nstrb) with row npair = c itself, so that the Gram entries (P, npair) are
// gamma+_P and (npair, npair) is |c|^2.  A tile of RD_BT determinants is
// built in shared memory ([RD_BT][R], R = npair + 1 rounded up to 4), then
// every thread adds the 4x4 blocks (bi <= bj) it owns.  FP32 mode: the tile
// sums are FP32 and they are added across tiles with Kahan compensation.
template <typename T, int NB>
__global__ void __launch_bounds__(RD_THREADS)
    k_rdm_partial(const int32_t* __restrict__ link, const int32_t* __restrict__ linkb, int nstrb,
                  int npair, const double* __restrict__ X, int N, int R, int nblk, int chunk,
                  int nchunk, double* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char rd_smem[];
  T* sD = reinterpret_cast<T*>(rd_smem);
  const int ch = blockIdx.x;
  const double* c = X + (int64_t)blockIdx.y * N;
  const int k_beg = ch * chunk, k_end = min(N, k_beg + chunk);
  const int nb4 = R / 4;
  int bi[NB], bj[NB];
  bool on[NB];
#pragma unroll
  for (int u = 0; u < NB; u++) {
    const int blk = threadIdx.x + u * RD_THREADS;
    on[u] = blk < nblk;
    int r = 0, rem = on[u] ? blk : 0;
    while (rem >= nb4 - r) {
      rem -= nb4 - r;
      r++;
    }
    bi[u] = 4 * r;
    bj[u] = 4 * (r + rem);
  }
  constexpr bool KAHAN = sizeof(T) == 4;
  T acc[NB][16], comp[NB][16];
#pragma unroll
  for (int u = 0; u < NB; u++)
#pragma unroll
    for (int e = 0; e < 16; e++) acc[u][e] = comp[u][e] = T(0);
  for (int k0 = k_beg; k0 < k_end; k0 += RD_BT) {
    for (int i = threadIdx.x; i < RD_BT * R; i += RD_THREADS) {
      const int kk = i % RD_BT, r = i / RD_BT;
      const int k = k0 + kk;
      T v = T(0);
      if (k < k_end && r <= npair) {
        if (r == npair) {
          v = (T)c[k];
        } else {
          const int a = k / nstrb, b = k - a * nstrb;
          const int32_t ta = link[(int64_t)a * npair + r], tb = linkb[(int64_t)b * npair + r];
          if (ta >= 0) {
            const T x = (T)c[(int64_t)(ta >> 1) * nstrb + b];
            v += (ta & 1) ? -x : x;
          }
          if (tb >= 0) {
            const T x = (T)c[(int64_t)a * nstrb + (tb >> 1)];
            v += (tb & 1) ? -x : x;
          }
        }
      }
      sD[kk * R + r] = v;
    }
    __syncthreads();
    T ts[NB][16];
#pragma unroll
    for (int u = 0; u < NB; u++)
#pragma unroll
      for (int e = 0; e < 16; e++) ts[u][e] = T(0);
#pragma unroll 4
    for (int kk = 0; kk < RD_BT; kk++) {
#pragma unroll
      for (int u = 0; u < NB; u++) {
        if (!on[u]) continue;
        T pa[4], pb[4];
        load4<T>(sD + kk * R + bi[u], pa);
        load4<T>(sD + kk * R + bj[u], pb);
#pragma unroll
        for (int ii = 0; ii < 4; ii++)
#pragma unroll
          for (int jj = 0; jj < 4; jj++) ts[u][ii * 4 + jj] = fma(pa[ii], pb[jj], ts[u][ii * 4 + jj]);
      }
    }
#pragma unroll
    for (int u = 0; u < NB; u++)
#pragma unroll
      for (int e = 0; e < 16; e++) {
        if (KAHAN) {
          const T y = ts[u][e] - comp[u][e];
          const T t = acc[u][e] + y;
          comp[u][e] = (t - acc[u][e]) - y;
          acc[u][e] = t;
        } else {
          acc[u][e] += ts[u][e];
        }
      }
    __syncthreads();
  }
  double* pp = part + ((int64_t)blockIdx.y * nchunk + ch) * nblk * 16;
#pragma unroll
  for (int u = 0; u < NB; u++) {
    if (!on[u]) continue;
    const int blk = threadIdx.x + u * RD_THREADS;
#pragma unroll
    for (int e = 0; e < 16; e++) pp[blk * 16 + e] = (double)acc[u][e] - (double)comp[u][e];
  }
}

// Sum of the chunk partials in chunk order, normalised by |c|^2, written as
// gamma+ (npair) then the upper triangle of Gamma' (row P holds Q = P..npair-1)
__global__ void k_rdm_finish(const double* __restrict__ part, int nchunk, int nblk, int npair,
                             int R, double* __restrict__ out, int64_t rs) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nblk * 16) return;
  const double* pb = part + (int64_t)blockIdx.y * nchunk * nblk * 16;
  const int nb4 = R / 4;
  auto row_start = [&](int r) { return r * nb4 - r * (r - 1) / 2; };
  const int dn = npair / 4;
  const int en = row_start(dn) * 16 + (npair % 4) * 5;
  double nrm = 0.0, s = 0.0;
  for (int ch = 0; ch < nchunk; ch++) {
    nrm += pb[(int64_t)ch * nblk * 16 + en];
    s += pb[(int64_t)ch * nblk * 16 + e];
  }
  const int blk = e / 16, ii = (e % 16) / 4, jj = e % 4;
  int r = 0;
  while (row_start(r + 1) <= blk) r++;
  const int P = 4 * r + ii, Q = 4 * (r + blk - row_start(r)) + jj;
  if (P > Q || Q > npair) return;
  double* o = out + (int64_t)blockIdx.y * rs;
  const double inv = 1.0 / nrm;
  if (Q == npair) {
    if (P < npair) o[P] = s * inv;
    return;
  }
  o[npair + P * npair - P * (P - 1) / 2 + (Q - P)] = s * inv;
}

__device__ __forceinline__ int pidx(int p, int q) {
  return p >= q ? p * (p + 1) / 2 + q : q * (q + 1) / 2 + p;
}

// Scatter w * (full-space RDM contributions) of one CASCI into dh (norb^2)
// and the unsymmetrised packed ERI gradient G (npair_g^2).
//  rel[nr]: the orbitals with non-zero RDM entries (core + active, sorted),
//  loc[nr]: their active index or -1 for core orbitals,
//  rdm: the packed active RDMs (gamma+, then the upper triangle of Gamma').
// Every thread owns distinct entries of dh and G, and the CASCIs are
// added one launch after another on one stream: plain read-modify-writes,
// in a fixed order.
__global__ void k_assemble(const int32_t* __restrict__ rel, const int32_t* __restrict__ loc, int nr,
                           int n_act, const double* __restrict__ rdm, double w, int norb,
                           int64_t npair_g, double* __restrict__ dh, double* __restrict__ G) {
  const int nrp = nr * (nr + 1) / 2;
  const int npa = n_act * (n_act + 1) / 2;
  const double* g1p = rdm;
  auto g2 = [&](int A, int Bq) -> double {
    if (A > Bq) {
      const int t = A;
      A = Bq;
      Bq = t;
    }
    return rdm[npa + (int64_t)A * npa - (int64_t)A * (A - 1) / 2 + (Bq - A)];
  };
  // full-space gamma between relevant orbitals i, j (local relevant indices)
  auto gam = [&](int i, int j) -> double {
    const int li = loc[i], lj = loc[j];
    if (li < 0 && lj < 0) return i == j ? 2.0 : 0.0;
    if (li < 0 || lj < 0) return 0.0;
    const double v = g1p[pidx(li, lj)];
    return li == lj ? v : 0.5 * v;
  };
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid < (int64_t)nr * nr) {
    const int i = (int)(tid / nr), j = (int)(tid % nr);
    dh[(int64_t)rel[i] * norb + rel[j]] += w * gam(i, j);
  }
  if (tid >= (int64_t)nrp * nrp) return;
  const int X = (int)(tid / nrp), Y = (int)(tid % nrp);
  int p = (int)((sqrtf(8.f * X + 1.f) - 1.f) * 0.5f);
  while (p * (p + 1) / 2 > X) p--;
  while ((p + 1) * (p + 2) / 2 <= X) p++;
  const int q = X - p * (p + 1) / 2;
  int r = (int)((sqrtf(8.f * Y + 1.f) - 1.f) * 0.5f);
  while (r * (r + 1) / 2 > Y) r--;
  while ((r + 1) * (r + 2) / 2 <= Y) r++;
  const int s = Y - r * (r + 1) / 2;
  const int ia[2] = {p, q}, ib[2] = {q, p}, ic[2] = {r, s}, id[2] = {s, r};
  const int n1 = p == q ? 1 : 2, n2 = r == s ? 1 : 2;
  const bool all_act = loc[p] >= 0 && loc[q] >= 0 && loc[r] >= 0 && loc[s] >= 0;
  double sum = 0.0;
  if (all_act) {
    // images of <E_ab E_cd> sum to Gamma'; subtract the d_bc gamma_ad images
    sum = g2(pidx(loc[p], loc[q]), pidx(loc[r], loc[s]));
    for (int u = 0; u < n1; u++)
      for (int v = 0; v < n2; v++)
        if (ib[u] == ic[v]) sum -= gam(ia[u], id[v]);
  } else {
    for (int u = 0; u < n1; u++)
      for (int v = 0; v < n2; v++) {
        const int a = ia[u], b = ib[u], cc = ic[v], d = id[v];
        sum += gam(a, b) * gam(cc, d) - 0.5 * gam(a, d) * gam(cc, b);
      }
  }
  if (sum != 0.0) {
    const int64_t P = pidx(rel[p], rel[q]), Q = pidx(rel[r], rel[s]);
    G[P * npair_g + Q] += w * 0.5 * sum;
  }
}

__global__ void k_symmetrize_out(const double* __restrict__ G, int64_t n, double* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * n) return;
  const int64_t i = t / n, j = t % n;
  out[t] = 0.5 * (G[i * n + j] + G[j * n + i]);
}

}  // namespace

// ------------------------------------------------------------------ host
void rdm_batch(mbe_ctx* ctx, const StringTables* tab, const StringTables* tabb, const double* X,
               int B, bool fp32, double* out) {
  if (B <= 0) return;
  const int npair = tab->npair, nstrb = tabb->nstr;
  const int N = tab->nstr * nstrb;
  const int R = (npair + 1 + 3) / 4 * 4;
  const int nb4 = R / 4, nblk = nb4 * (nb4 + 1) / 2;
  if (nblk > 2 * RD_THREADS) throw MbeError{MBE_EINVAL, "active space too large for the RDM kernel"};
  int nsm = 0;
  CU_CHECK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
  // about two CTAs per SM over the batch, at least 8 tiles per chunk
  int nchunk = std::max(1, (2 * nsm + B - 1) / B);
  nchunk = std::min(nchunk, std::max(1, N / (8 * RD_BT)));
  int chunk = (N + nchunk - 1) / nchunk;
  chunk = (chunk + RD_BT - 1) / RD_BT * RD_BT;
  nchunk = (N + chunk - 1) / chunk;
  DevBuf<double> part(&ctx->pool, (size_t)B * nchunk * nblk * 16);
  cudaStream_t st = ctx->stream;
  const dim3 grid((unsigned)nchunk, (unsigned)B);
  const size_t smem = (size_t)RD_BT * R * (fp32 ? 4 : 8);
  const int32_t* link = tab->link.ptr;
  const int32_t* linkb = tabb->link.ptr;
  if (fp32) {
    if (nblk <= RD_THREADS)
      k_rdm_partial<float, 1><<<grid, RD_THREADS, smem, st>>>(
          link, linkb, nstrb, npair, X, N, R, nblk, chunk, nchunk, part.ptr);
    else
      k_rdm_partial<float, 2><<<grid, RD_THREADS, smem, st>>>(
          link, linkb, nstrb, npair, X, N, R, nblk, chunk, nchunk, part.ptr);
  } else {
    if (nblk <= RD_THREADS)
      k_rdm_partial<double, 1><<<grid, RD_THREADS, smem, st>>>(
          link, linkb, nstrb, npair, X, N, R, nblk, chunk, nchunk, part.ptr);
    else
      k_rdm_partial<double, 2><<<grid, RD_THREADS, smem, st>>>(
          link, linkb, nstrb, npair, X, N, R, nblk, chunk, nchunk, part.ptr);
  }
  CU_LAUNCH_CHECK();
  k_rdm_finish<<<dim3((unsigned)((nblk * 16 + 255) / 256), (unsigned)B), 256, 0, st>>>(
      part.ptr, nchunk, nblk, npair, R, out, rdm_size(npair));
  CU_LAUNCH_CHECK();
}

int backward_run(mbe_ctx* ctx, double scale, double* dh_host, double* deri_host) {
  if (!ctx->opt.keep_ci) throw MbeError{MBE_ESTATE, "energy backward needs keep_ci = 1"};
  if (!ctx->have_ref) throw MbeError{MBE_ESTATE, "no reference space set"};
  cudaStream_t st = ctx->stream;
  DevPool* P = &ctx->pool;
  const int norb = ctx->norb;
  const int64_t npg = ctx->npair_g;
  HashTable& H = ctx->hash;
  // ---- MBE coefficients of every processed tuple (slots of the hash)
  DevBuf<int32_t> coef(P, H.cap), cref(P, 1), err(P, 1);
  CU_CHECK(cudaMemsetAsync(coef.ptr, 0, sizeof(int32_t) * H.cap, st));
  CU_CHECK(cudaMemsetAsync(cref.ptr, 0, sizeof(int32_t), st));
  CU_CHECK(cudaMemsetAsync(err.ptr, 0, sizeof(int32_t), st));
  std::vector<std::unique_ptr<DevBuf<int32_t>>> tbufs;
  for (const OrderRec& r : ctx->history) {
    const int64_t nt = (int64_t)r.inc.size();
    if (!nt) continue;
    tbufs.push_back(std::make_unique<DevBuf<int32_t>>(P, r.tuples.size()));
    CU_CHECK(cudaMemcpyAsync(tbufs.back()->ptr, r.tuples.data(), sizeof(int32_t) * r.tuples.size(),
                             cudaMemcpyHostToDevice, st));
    mbe_coef_launch(ctx, tbufs.back()->ptr, r.order, nt, coef.ptr, cref.ptr, err.ptr);
  }
  int32_t e = 0, cr = 0;
  CU_CHECK(cudaMemcpyAsync(&e, err.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CU_CHECK(cudaMemcpyAsync(&cr, cref.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  // coefficient of each kept RDM: look its key up on the host mirror
  std::vector<int32_t> coef_h(H.cap);
  std::vector<unsigned long long> keys_h(2 * H.cap);
  std::vector<int32_t> state_h(H.cap);
  if (H.cap) {
    CU_CHECK(cudaMemcpyAsync(coef_h.data(), coef.ptr, sizeof(int32_t) * H.cap,
                             cudaMemcpyDeviceToHost, st));
    CU_CHECK(cudaMemcpyAsync(keys_h.data(), H.keys.ptr, sizeof(unsigned long long) * 2 * H.cap,
                             cudaMemcpyDeviceToHost, st));
    CU_CHECK(cudaMemcpyAsync(state_h.data(), H.state.ptr, sizeof(int32_t) * H.cap,
                             cudaMemcpyDeviceToHost, st));
  }
  CU_CHECK(cudaStreamSynchronize(st));
  tbufs.clear();
  if (e) throw MbeError{MBE_ELOOKUP, "a subtuple is missing from the hash"};
  cr += 1;   // the empty tuple itself
  const int share = ctx->opt.backward_share;
  std::map<std::pair<unsigned long long, unsigned long long>, int32_t> kc;
  for (int64_t s = 0; s < H.cap; s++)
    if (state_h[s]) kc[{keys_h[2 * s], keys_h[2 * s + 1]}] = coef_h[s];

  // ---- the weighted CASCIs: relevant orbitals of each, packed for one copy
  struct Job {
    int64_t off;
    int nr, n_act;
    const double* rdm;
    double w;
  };
  std::vector<Job> jobs;
  std::vector<int32_t> relloc;   // per job: rel[nr] then loc[nr]
  std::vector<bool> is_act(norb, false);
  auto add_job = [&](const std::vector<int32_t>& tuple, const double* rdm, double w) {
    std::vector<int> act(ctx->ref.begin(), ctx->ref.end());
    for (int o : tuple) act.push_back(o);
    std::sort(act.begin(), act.end());
    std::fill(is_act.begin(), is_act.end(), false);
    for (int a : act) is_act[a] = true;
    std::vector<int32_t> rel, loc;
    for (int o = 0; o < norb; o++) {
      if (is_act[o]) {
        rel.push_back(o);
        loc.push_back((int32_t)(std::lower_bound(act.begin(), act.end(), o) - act.begin()));
      } else if (o < ctx->nocc) {
        rel.push_back(o);
        loc.push_back(-1);
      }
    }
    if (rel.empty()) return;
    if (!act.empty() && !rdm) throw MbeError{MBE_ESTATE, "kept RDMs missing"};
    jobs.push_back({(int64_t)relloc.size(), (int)rel.size(), (int)act.size(), rdm, w});
    relloc.insert(relloc.end(), rel.begin(), rel.end());
    relloc.insert(relloc.end(), loc.begin(), loc.end());
  };
  if (cr != 0 && share != 1) {
    if (ctx->ref.empty()) add_job({}, nullptr, scale * cr);   // closed-shell core only
    else if (ctx->kept_ref) add_job({}, ctx->ref_ci.rdm, scale * cr);
    else throw MbeError{MBE_ESTATE, "reference RDMs missing (set keep_ci before mbe_set_reference)"};
  }
  for (const KeptRdm& k : ctx->kept) {
    unsigned long long k0 = 0, k1 = 0;
    for (int o : k.tuple) {
      if (o < 64) k0 |= 1ull << o; else k1 |= 1ull << (o - 64);
    }
    auto it = kc.find({k0, k1});
    if (it == kc.end()) continue;   // solved but not processed by mbe_increments
    if (it->second != 0) add_job(k.tuple, k.rdm, scale * it->second);
    it->second = 0;                 // done
  }
  if (share == 0)
    for (const auto& kv : kc)
      if (kv.second != 0)
        throw MbeError{MBE_ESTATE, "the RDMs of a tuple of the expansion are not held (keep_ci was 0?)"};

  DevBuf<double> dh(P, (size_t)norb * norb), G(P, (size_t)(npg * npg));
  CU_CHECK(cudaMemsetAsync(dh.ptr, 0, sizeof(double) * norb * norb, st));
  CU_CHECK(cudaMemsetAsync(G.ptr, 0, sizeof(double) * npg * npg, st));
  DevBuf<int32_t> rl(P, std::max<size_t>(1, relloc.size()));
  if (!relloc.empty())
    CU_CHECK(cudaMemcpyAsync(rl.ptr, relloc.data(), sizeof(int32_t) * relloc.size(),
                             cudaMemcpyHostToDevice, st));
  // one launch per CASCI, in a fixed order on one stream (no host waits)
  for (const Job& j : jobs) {
    const int64_t nrp = (int64_t)j.nr * (j.nr + 1) / 2;
    const int64_t nth = std::max<int64_t>(nrp * nrp, (int64_t)j.nr * j.nr);
    k_assemble<<<(unsigned)((nth + 255) / 256), 256, 0, st>>>(
        rl.ptr + j.off, rl.ptr + j.off + j.nr, j.nr, j.n_act, j.rdm, j.w, norb, npg, dh.ptr, G.ptr);
    CU_LAUNCH_CHECK();
  }
  DevBuf<double> Gs(P, (size_t)(npg * npg));
  k_symmetrize_out<<<(unsigned)((npg * npg + 255) / 256), 256, 0, st>>>(G.ptr, npg, Gs.ptr);
  CU_LAUNCH_CHECK();
  CU_CHECK(cudaMemcpyAsync(dh_host, dh.ptr, sizeof(double) * norb * norb, cudaMemcpyDeviceToHost, st));
  CU_CHECK(cudaMemcpyAsync(deri_host, Gs.ptr, sizeof(double) * npg * npg, cudaMemcpyDeviceToHost, st));
  CU_CHECK(cudaStreamSynchronize(st));
  return MBE_OK;
}
