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
#include "mbe_internal.cuh"
#include <algorithm>
#include <cmath>

namespace {

// gamma+_P = sum_K c_K D_P(K) and Gamma'_PQ = sum_K D_P(K) D_Q(K), one 16x16
// tile of (P, Q) per block, FP64 with fixed-order reductions
__global__ void k_rdm_packed(const double* __restrict__ D, const double* __restrict__ c, int npair,
                             int64_t N, double* __restrict__ g1p, double* __restrict__ g2p) {
  const int P0 = blockIdx.x * 16, Q0 = blockIdx.y * 16;
  __shared__ double sP[16][65], sQ[16][65], sc[64];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc = 0.0, acc1 = 0.0;
  for (int64_t k0 = 0; k0 < N; k0 += 64) {
    for (int i = threadIdx.x; i < 16 * 64; i += 256) {
      const int r = i >> 6, kk = i & 63;
      const int64_t k = k0 + kk;
      sP[r][kk] = (P0 + r < npair && k < N) ? D[(int64_t)(P0 + r) * N + k] : 0.0;
      sQ[r][kk] = (Q0 + r < npair && k < N) ? D[(int64_t)(Q0 + r) * N + k] : 0.0;
    }
    if (threadIdx.x < 64) sc[threadIdx.x] = (k0 + threadIdx.x < N) ? c[k0 + threadIdx.x] : 0.0;
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 64; kk++) {
      acc = fma(sP[ty][kk], sQ[tx][kk], acc);
      if (blockIdx.y == 0 && tx == 0) acc1 = fma(sP[ty][kk], sc[kk], acc1);
    }
    __syncthreads();
  }
  if (P0 + ty < npair && Q0 + tx < npair) g2p[(int64_t)(P0 + ty) * npair + Q0 + tx] = acc;
  if (blockIdx.y == 0 && tx == 0 && P0 + ty < npair) g1p[P0 + ty] = acc1;
}

__device__ __forceinline__ int pidx(int p, int q) {
  return p >= q ? p * (p + 1) / 2 + q : q * (q + 1) / 2 + p;
}

// Scatter w * (full-space RDM contributions) of one CASCI into dh (norb^2)
// and the unsymmetrised packed ERI gradient G (npair_g^2).
//  rel[nr]: the orbitals with non-zero RDM entries (core + active, sorted),
//  loc[nr]: their active index or -1 for core orbitals.
__global__ void k_assemble(const int32_t* __restrict__ rel, const int32_t* __restrict__ loc, int nr,
                           int n_act, const double* __restrict__ g1p,
                           const double* __restrict__ g2p, double w, int norb, int64_t npair_g,
                           double* __restrict__ dh, double* __restrict__ G) {
  const int nrp = nr * (nr + 1) / 2;
  const int npa = n_act * (n_act + 1) / 2;
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
    atomicAdd(&dh[(int64_t)rel[i] * norb + rel[j]], w * gam(i, j));
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
    sum = g2p[(int64_t)pidx(loc[p], loc[q]) * npa + pidx(loc[r], loc[s])];
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
    atomicAdd(&G[P * npair_g + Q], w * 0.5 * sum);
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
  for (const OrderRec& r : ctx->history) {
    const int64_t nt = (int64_t)r.inc.size();
    if (!nt) continue;
    DevBuf<int32_t> tb(P, r.tuples.size());
    CU_CHECK(cudaMemcpyAsync(tb.ptr, r.tuples.data(), sizeof(int32_t) * r.tuples.size(),
                             cudaMemcpyHostToDevice, st));
    mbe_coef_launch(ctx, tb.ptr, r.order, nt, coef.ptr, cref.ptr, err.ptr);
    CU_CHECK(cudaStreamSynchronize(st));
  }
  int32_t e = 0, cr = 0;
  CU_CHECK(cudaMemcpyAsync(&e, err.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CU_CHECK(cudaMemcpyAsync(&cr, cref.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  // coefficient of each kept CI vector: look its key up on the host mirror
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
  if (e) throw MbeError{MBE_ELOOKUP, "a subtuple is missing from the hash"};
  cr += 1;   // the empty tuple itself
  const int share = ctx->opt.backward_share;
  std::map<std::pair<unsigned long long, unsigned long long>, int32_t> kc;
  for (int64_t s = 0; s < H.cap; s++)
    if (state_h[s]) kc[{keys_h[2 * s], keys_h[2 * s + 1]}] = coef_h[s];

  DevBuf<double> dh(P, (size_t)norb * norb), G(P, (size_t)(npg * npg));
  CU_CHECK(cudaMemsetAsync(dh.ptr, 0, sizeof(double) * norb * norb, st));
  CU_CHECK(cudaMemsetAsync(G.ptr, 0, sizeof(double) * npg * npg, st));

  // one CASCI (active space ref + tuple, CI vector c) with weight w
  auto add_casci = [&](const std::vector<int32_t>& tuple, int nsig, const std::vector<double>& c,
                       double w) {
    std::vector<int> act(ctx->ref.begin(), ctx->ref.end());
    for (int o : tuple) act.push_back(o);
    std::sort(act.begin(), act.end());
    const int n = (int)act.size();
    // relevant orbitals: inactive core + active, with their active index
    std::vector<int32_t> rel, loc;
    std::vector<bool> is_act(norb, false);
    for (int a : act) is_act[a] = true;
    for (int o = 0; o < norb; o++) {
      if (is_act[o]) {
        rel.push_back(o);
        loc.push_back((int32_t)(std::lower_bound(act.begin(), act.end(), o) - act.begin()));
      } else if (o < ctx->nocc) {
        rel.push_back(o);
        loc.push_back(-1);
      }
    }
    const int nr = (int)rel.size();
    if (nr == 0) return;
    DevBuf<int32_t> reld(P, nr), locd(P, nr);
    CU_CHECK(cudaMemcpyAsync(reld.ptr, rel.data(), sizeof(int32_t) * nr, cudaMemcpyHostToDevice, st));
    CU_CHECK(cudaMemcpyAsync(locd.ptr, loc.data(), sizeof(int32_t) * nr, cudaMemcpyHostToDevice, st));
    int npa = 0;
    DevBuf<double> g1p, g2p;
    if (n > 0) {
      const StringTables* tab = get_tables(ctx, n, nsig);
      npa = tab->npair;
      const int64_t N = (int64_t)tab->nstr * tab->nstr;
      if ((int64_t)c.size() != N) throw MbeError{MBE_ESTATE, "kept CI vector has the wrong length"};
      // normalised copy of the CI vector
      double nn = 0.0;
      for (double v : c) nn += v * v;
      if (!(nn > 0.0)) throw MbeError{MBE_ESTATE, "kept CI vector is zero"};
      const double inv = 1.0 / std::sqrt(nn);
      std::vector<double> cn(c.size());
      for (size_t i = 0; i < c.size(); i++) cn[i] = c[i] * inv;
      DevBuf<double> cd(P, N), D(P, (size_t)npa * N);
      g1p.reset(P, npa);
      g2p.reset(P, (size_t)npa * npa);
      CU_CHECK(cudaMemcpyAsync(cd.ptr, cn.data(), sizeof(double) * N, cudaMemcpyHostToDevice, st));
      gather_d_fp64(ctx, tab, cd.ptr, D.ptr);
      dim3 gr((npa + 15) / 16, (npa + 15) / 16);
      k_rdm_packed<<<gr, 256, 0, st>>>(D.ptr, cd.ptr, npa, N, g1p.ptr, g2p.ptr);
      CU_LAUNCH_CHECK();
      CU_CHECK(cudaStreamSynchronize(st));
    }
    const int64_t nrp = (int64_t)nr * (nr + 1) / 2;
    const int64_t nth = std::max<int64_t>(nrp * nrp, (int64_t)nr * nr);
    k_assemble<<<(unsigned)((nth + 255) / 256), 256, 0, st>>>(reld.ptr, locd.ptr, nr, n, g1p.ptr,
                                                              g2p.ptr, w, norb, npg, dh.ptr, G.ptr);
    CU_LAUNCH_CHECK();
    CU_CHECK(cudaStreamSynchronize(st));
  };

  if (cr != 0 && share != 1) {
    if (ctx->ref.empty()) add_casci({}, 0, {}, scale * cr);   // closed-shell core only
    else if (ctx->kept_ref) add_casci({}, ctx->ref_ci.nsig, ctx->ref_ci.c, scale * cr);
    else throw MbeError{MBE_ESTATE, "reference CI vector missing (set keep_ci before mbe_set_reference)"};
  }
  for (const KeptCI& k : ctx->kept) {
    unsigned long long k0 = 0, k1 = 0;
    for (int o : k.tuple) {
      if (o < 64) k0 |= 1ull << o; else k1 |= 1ull << (o - 64);
    }
    auto it = kc.find({k0, k1});
    if (it == kc.end()) continue;   // solved but not processed by mbe_increments
    if (it->second != 0) add_casci(k.tuple, k.nsig, k.c, scale * it->second);
    it->second = 0;                 // done
  }
  if (share == 0)
    for (const auto& kv : kc)
      if (kv.second != 0)
        throw MbeError{MBE_ESTATE, "a CI vector of the expansion is not held (keep_ci was 0?)"};
  DevBuf<double> Gs(P, (size_t)(npg * npg));
  k_symmetrize_out<<<(unsigned)((npg * npg + 255) / 256), 256, 0, st>>>(G.ptr, npg, Gs.ptr);
  CU_LAUNCH_CHECK();
  CU_CHECK(cudaMemcpyAsync(dh_host, dh.ptr, sizeof(double) * norb * norb, cudaMemcpyDeviceToHost, st));
  CU_CHECK(cudaMemcpyAsync(deri_host, Gs.ptr, sizeof(double) * npg * npg, cudaMemcpyDeviceToHost, st));
  CU_CHECK(cudaStreamSynchronize(st));
  return MBE_OK;
}
