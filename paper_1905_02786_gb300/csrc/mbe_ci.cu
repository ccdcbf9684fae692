// CASCI building blocks of one bin of tuples (same active size n and same
// number of active electrons per spin nsig):
//   K1  string enumeration and the per-(string, orbital pair) link table
//   K2  effective integrals of each tuple (inactive-core fold, Sec. 2/Fig. 2)
//   K3  diagonal of H_active + shift * S^2 (Davidson preconditioner)
//   K4  FP64 string-driven sigma vector: gather D, (kl|ij) contraction, pull
//       scatter, plus the S^2 spin shift
//
// Sigma vector (Knowles & Handy, Chem. Phys. Lett. 111, 315 (1984); Olsen
// et al., J. Chem. Phys. 89, 2185 (1988)): with h'_pq = h_pq - 1/2 sum_r
// (pr|rq) and g'_{pq,rs} = (pq|rs) + (h'_pq d_rs + d_pq h'_rs)/N the active
// Hamiltonian is H = 1/2 sum_{PQ} g'_{PQ} E+_P E+_Q over packed pairs
// P = (p >= q), E+_P = E_pq + E_qp (E_pp on the diagonal).  Hence
//   D_P(K)  = sum_J <K|E+_P|J> c_J            (gather)
//   F_P(K)  = sum_Q g'_{PQ} D_Q(K)            (contraction)
//   sigma_I = 1/2 sum_P sum_K <I|E+_P|K> F_P(K)   (pull scatter)
// E+_P acting on one spin string has at most one non-zero matrix element
// per string, which the link table stores.
#include "mbe_internal.cuh"

namespace {

__constant__ int c_binom[33][33];

bool g_binom_ready[MBE_MAX_DEVICES] = {false};

// the binomial table is copied with a synchronous cudaMemcpyToSymbol on the
// first use on a device (it waits for the device once)
void ensure_binom(int device) {
  once_per_device(g_binom_ready, device, [] {
    int tab[33][33];
    for (int n = 0; n <= 32; n++)
      for (int k = 0; k <= 32; k++) {
        if (k == 0) tab[n][k] = 1;
        else if (n == 0) tab[n][k] = 0;
        else {
          long long v = (long long)tab[n - 1][k - 1] + tab[n - 1][k];
          tab[n][k] = v > 0x7fffffff ? 0x7fffffff : (int)v;
        }
      }
    CU_CHECK(cudaMemcpyToSymbol(c_binom, tab, sizeof(tab)));
  });
}

// colexicographic rank of a k-subset bit mask = its position when all
// k-subsets are sorted by integer value
__device__ __forceinline__ int mask_rank(uint32_t m) {
  int r = 0, i = 1;
  while (m) {
    int p = __ffs(m) - 1;
    r += c_binom[p][i];
    i++;
    m &= m - 1;
  }
  return r;
}

__device__ uint32_t mask_unrank(int r, int n, int k) {
  uint32_t m = 0;
  for (int i = k; i >= 1; i--) {
    int p = i - 1;
    while (p + 1 < n && c_binom[p + 1][i] <= r) p++;
    m |= 1u << p;
    r -= c_binom[p][i];
  }
  return m;
}

__global__ void k_strings(uint32_t* masks, int nstr, int n, int k) {
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I < nstr) masks[I] = mask_unrank(I, n, k);
}

__global__ void k_link(const uint32_t* masks, int32_t* link, int nstr, int n) {
  int npair = n * (n + 1) / 2;
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nstr * npair) return;
  int I = (int)(t / npair), P = (int)(t % npair);
  int p = (int)((sqrtf(8.f * P + 1.f) - 1.f) * 0.5f);
  while (p * (p + 1) / 2 > P) p--;
  while ((p + 1) * (p + 2) / 2 <= P) p++;
  int q = P - p * (p + 1) / 2;
  uint32_t m = masks[I];
  int32_t v = -1;
  int bp = (m >> p) & 1, bq = (m >> q) & 1;
  if (p == q) {
    if (bp) v = I << 1;
  } else if (bp != bq) {
    uint32_t J = m ^ (1u << p) ^ (1u << q);
    // orbitals strictly between q and p (p > q) decide the sign
    uint32_t between = (m & ((1u << p) - 1u)) & ~((2u << q) - 1u);
    int neg = __popc(between) & 1;
    v = (mask_rank(J) << 1) | neg;
  }
  link[t] = v;
}

}  // namespace

int64_t string_count(int n, int nsig) {
  long long nstr = 1;
  for (int i = 0; i < nsig; i++) nstr = nstr * (n - i) / (i + 1);
  return nstr;
}

void launch_string_tables(mbe_ctx* ctx, int n, int nsig, int nstr, uint32_t* masks,
                          int32_t* link) {
  ensure_binom(ctx->device);
  k_strings<<<(nstr + 255) / 256, 256, 0, ctx->stream>>>(masks, nstr, n, nsig);
  CU_LAUNCH_CHECK();
  const int64_t tot = (int64_t)nstr * (n * (n + 1) / 2);
  k_link<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(masks, link, nstr, n);
  CU_LAUNCH_CHECK();
}

void build_string_tables(mbe_ctx* ctx, StringTables* t) {
  const int64_t nstr = string_count(t->n, t->nsig);
  if (nstr > (1 << 28)) throw MbeError{MBE_EINVAL, "string space too large"};
  t->nstr = (int)nstr;
  t->npair = t->n * (t->n + 1) / 2;
  t->masks.reset(&ctx->pool, t->nstr);
  t->link.reset(&ctx->pool, (size_t)t->nstr * t->npair);
  launch_string_tables(ctx, t->n, t->nsig, t->nstr, t->masks.ptr, t->link.ptr);
}

// ------------------------------------------------------------------ K2
namespace {

__device__ __forceinline__ int64_t gpair(int p, int q) {
  return p >= q ? (int64_t)p * (p + 1) / 2 + q : (int64_t)q * (q + 1) / 2 + p;
}

// One CTA per tuple.  act: n sorted global orbital ids.
__global__ void k_effints(const double* __restrict__ h, const double* __restrict__ eri,
                          int norb, int nocc, int npair_g, const int32_t* __restrict__ act_all,
                          int n, int nel, double* ecore_out, double* heff_out, double* hp_out,
                          double* gp_out, double* jk_out) {
  const int b = blockIdx.x;
  const int32_t* act = act_all + (int64_t)b * n;
  extern __shared__ double sm[];
  double* s_heff = sm;            // n*n
  double* s_hp = sm + n * n;      // n*n
  __shared__ int s_core[MBE_MAX_NORB];
  __shared__ int s_ncore;
  __shared__ int s_act[MBE_MAX_ACT];
  if (threadIdx.x == 0) {
    int nc = 0, j = 0;
    for (int i = 0; i < nocc; i++) {
      while (j < n && act[j] < i) j++;
      if (!(j < n && act[j] == i)) s_core[nc++] = i;
    }
    s_ncore = nc;
  }
  if (threadIdx.x < n) s_act[threadIdx.x] = act[threadIdx.x];
  __syncthreads();
  const int nc = s_ncore;
  const int64_t NP = npair_g;
  // inactive-core energy (Fig. 2: occupied orbitals outside the active space
  // stay doubly occupied): sum 2 h_ii + sum_ij [2 (ii|jj) - (ij|ji)]
  if (threadIdx.x == 0) {
    double e = 0.0;
    for (int x = 0; x < nc; x++) {
      int i = s_core[x];
      e += 2.0 * h[(int64_t)i * norb + i];
    }
    double e2 = 0.0;
    for (int x = 0; x < nc; x++)
      for (int y = 0; y < nc; y++) {
        int i = s_core[x], j = s_core[y];
        e2 += 2.0 * eri[gpair(i, i) * NP + gpair(j, j)] - eri[gpair(i, j) * NP + gpair(j, i)];
      }
    ecore_out[b] = e + e2;
  }
  // h_eff_pq = h_pq + sum_i [2 (pq|ii) - (pi|iq)]
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    int p = t / n, q = t % n;
    int P = s_act[p], Q = s_act[q];
    double v = h[(int64_t)P * norb + Q];
    for (int x = 0; x < nc; x++) {
      int i = s_core[x];
      v += 2.0 * eri[gpair(P, Q) * NP + gpair(i, i)] - eri[gpair(P, i) * NP + gpair(i, Q)];
    }
    s_heff[t] = v;
    heff_out[(int64_t)b * n * n + t] = v;
    jk_out[(int64_t)b * 2 * n * n + t] = eri[gpair(P, P) * NP + gpair(Q, Q)];
    jk_out[(int64_t)b * 2 * n * n + n * n + t] = eri[gpair(P, Q) * NP + gpair(Q, P)];
  }
  __syncthreads();
  // h'_pq = h_eff_pq - 1/2 sum_r (pr|rq), r over the active orbitals
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    int p = t / n, q = t % n;
    int P = s_act[p], Q = s_act[q];
    double v = 0.0;
    for (int r = 0; r < n; r++) {
      int R = s_act[r];
      v += eri[gpair(P, R) * NP + gpair(R, Q)];
    }
    s_hp[t] = s_heff[t] - 0.5 * v;
    hp_out[(int64_t)b * n * n + t] = s_hp[t];
  }
  __syncthreads();
  // g'_{PQ} = (pq|rs) + (h'_pq d_rs + d_pq h'_rs) / N_active, N_active = nel
  // active electrons of both spins (sum_r E_rr = N_active on the space)
  const int npair = n * (n + 1) / 2;
  const double inv = nel > 0 ? 1.0 / nel : 0.0;
  for (int t = threadIdx.x; t < npair * npair; t += blockDim.x) {
    int P = t / npair, Q = t % npair;
    int p = (int)((sqrt(8.0 * P + 1.0) - 1.0) * 0.5);
    while (p * (p + 1) / 2 > P) p--;
    while ((p + 1) * (p + 2) / 2 <= P) p++;
    int q = P - p * (p + 1) / 2;
    int r = (int)((sqrt(8.0 * Q + 1.0) - 1.0) * 0.5);
    while (r * (r + 1) / 2 > Q) r--;
    while ((r + 1) * (r + 2) / 2 <= Q) r++;
    int s = Q - r * (r + 1) / 2;
    double v = eri[gpair(s_act[p], s_act[q]) * NP + gpair(s_act[r], s_act[s])];
    if (r == s) v += s_hp[p * n + q] * inv;
    if (p == q) v += s_hp[r * n + s] * inv;
    gp_out[(int64_t)b * npair * npair + t] = v;
  }
}

}  // namespace

void launch_effints_raw(mbe_ctx* ctx, const int32_t* act, int B, int n, int nel, double* ecore,
                        double* heff, double* hp, double* gp, double* jk) {
  size_t smem = 2 * sizeof(double) * n * n;
  k_effints<<<B, 256, smem, ctx->stream>>>(ctx->h.ptr, ctx->eri.ptr, ctx->norb, ctx->nocc,
                                           ctx->npair_g, act, n, nel, ecore, heff, hp, gp, jk);
  CU_LAUNCH_CHECK();
}

void launch_effints(mbe_ctx* ctx, BinProblem& bp) {
  const int n = bp.n, B = bp.B;
  bp.ecore.reset(&ctx->pool, B);
  bp.heff.reset(&ctx->pool, (size_t)B * n * n);
  bp.hp.reset(&ctx->pool, (size_t)B * n * n);
  bp.gp.reset(&ctx->pool, (size_t)B * bp.npair * bp.npair);
  bp.jk.reset(&ctx->pool, (size_t)B * 2 * n * n);
  const int nel = bp.nsig + (bp.nsigb < 0 ? bp.nsig : bp.nsigb);
  launch_effints_raw(ctx, bp.act.ptr, B, n, nel, bp.ecore.ptr, bp.heff.ptr, bp.hp.ptr,
                     bp.gp.ptr, bp.jk.ptr);
}

// ------------------------------------------------------------------ K3
namespace {

// energy of one spin string with itself: sum h_pp + 1/2 sum_{pq} (J - K)
__device__ __forceinline__ double string_self(uint32_t m, const double* heff, const double* J,
                                              const double* K, int n) {
  double e = 0.0, e2 = 0.0;
  for (int p = 0; p < n; p++) {
    if (!((m >> p) & 1)) continue;
    e += heff[p * n + p];
    for (int q = 0; q < n; q++)
      if ((m >> q) & 1) e2 += J[p * n + q] - K[p * n + q];
  }
  return e + 0.5 * e2;
}

// <Ia Ib| H_active + shift S^2 |Ia Ib>, computed symmetrically in (Ia, Ib).
// alpha strings masks[nstr], beta strings masksb[nstrb] (the same table for
// a closed shell); <S^2> diagonal = (beta-only orbitals) + Ms(Ms+1) (msms).
__global__ void k_hdiag(const uint32_t* __restrict__ masks, const uint32_t* __restrict__ masksb,
                        int nstr, int nstrb, int n, int nsigb, double msms,
                        const double* __restrict__ heff_all, const double* __restrict__ jk_all,
                        double shift, double* hd_all) {
  const int b = blockIdx.y;
  extern __shared__ double sm[];
  double* s_heff = sm;
  double* s_J = sm + n * n;
  double* s_K = sm + 2 * n * n;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    s_heff[t] = heff_all[(int64_t)b * n * n + t];
    s_J[t] = jk_all[(int64_t)b * 2 * n * n + t];
    s_K[t] = jk_all[(int64_t)b * 2 * n * n + n * n + t];
  }
  __syncthreads();
  const int64_t ndet = (int64_t)nstr * nstrb;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ndet;
       i += (int64_t)gridDim.x * blockDim.x) {
    int ia = (int)(i / nstrb), ib = (int)(i % nstrb);
    uint32_t ma = masks[ia], mb = masksb[ib];
    double ea = string_self(ma, s_heff, s_J, s_K, n);
    double eb = string_self(mb, s_heff, s_J, s_K, n);
    double cross = 0.0;
    for (int p = 0; p < n; p++) {
      int ap = (ma >> p) & 1, bpp = (mb >> p) & 1;
      if (ap & bpp) cross += s_J[p * n + p];
      for (int q = 0; q < p; q++) {
        int w = (ap & ((mb >> q) & 1)) + (((ma >> q) & 1) & bpp);
        if (w) cross += w * s_J[p * n + q];
      }
    }
    int ndocc = __popc(ma & mb);
    hd_all[(int64_t)b * ndet + i] = (ea + eb) + cross + shift * ((double)(nsigb - ndocc) + msms);
  }
}

}  // namespace

void launch_hdiag(mbe_ctx* ctx, BinProblem& bp, double spin_shift, double* hd) {
  const int n = bp.n;
  size_t smem = 3 * sizeof(double) * n * n;
  int64_t blocks = (bp.ndet + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  dim3 grid((unsigned)blocks, bp.B);
  k_hdiag<<<grid, 256, smem, ctx->stream>>>(bp.tab->masks.ptr, bp.tabb->masks.ptr, bp.nstr,
                                            bp.nstrb, n, bp.nsigb, bp.msms(), bp.heff.ptr,
                                            bp.jk.ptr, spin_shift, hd);
  CU_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ K4
namespace {

// D[b][P][Ia*nstr+Ib] = s_a C(Ja, Ib) + s_b C(Ia, Jb)
__global__ void k_gather_fp64(const int32_t* __restrict__ link, const int32_t* __restrict__ linkb,
                              int nstr, int nstrb, int npair,
                              const double* __restrict__ c, int64_t c_stride,
                              const int32_t* __restrict__ active, const int32_t* __restrict__ bmap,
                              double* __restrict__ D) {
  const int bl = blockIdx.y;                 // local index in the sub-batch
  const int b = bmap[bl];
  if (active && !active[b]) return;
  const double* cb = c + (int64_t)b * c_stride;
  const int64_t ndet = (int64_t)nstr * nstrb;
  double* Db = D + (int64_t)bl * npair * ndet;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ndet;
       i += (int64_t)gridDim.x * blockDim.x) {
    int ia = (int)(i / nstrb), ib = (int)(i % nstrb);
    const int32_t* la = link + (int64_t)ia * npair;
    const int32_t* lb = linkb + (int64_t)ib * npair;
    for (int P = 0; P < npair; P++) {
      double v = 0.0;
      int32_t ta = la[P], tb = lb[P];
      if (ta >= 0) {
        double x = cb[(int64_t)(ta >> 1) * nstrb + ib];
        v += (ta & 1) ? -x : x;
      }
      if (tb >= 0) {
        double x = cb[(int64_t)ia * nstrb + (tb >> 1)];
        v += (tb & 1) ? -x : x;
      }
      Db[(int64_t)P * ndet + i] = v;
    }
  }
}

// E[b][P][k] = sum_Q g'[b][P][Q] D[b][Q][k]: FP64 tiles of all rows x 64 columns
constexpr int GT_N = 64;
__global__ void __launch_bounds__(256) k_contract_fp64(const double* __restrict__ gp_all, int npair,
                                                       const double* __restrict__ D, int64_t ndet,
                                                       const int32_t* __restrict__ active,
                                                       const int32_t* __restrict__ bmap,
                                                       double* __restrict__ E) {
  const int bl = blockIdx.y;
  const int b = bmap[bl];
  if (active && !active[b]) return;
  extern __shared__ double sm[];
  double* s_g = sm;                          // npair * npair
  double* s_d = sm + npair * npair;          // npair * GT_N
  const double* g = gp_all + (int64_t)b * npair * npair;
  for (int t = threadIdx.x; t < npair * npair; t += blockDim.x) s_g[t] = g[t];
  const double* Db = D + (int64_t)bl * npair * ndet;
  double* Eb = E + (int64_t)bl * npair * ndet;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  for (int64_t col0 = (int64_t)blockIdx.x * GT_N; col0 < ndet; col0 += (int64_t)gridDim.x * GT_N) {
    __syncthreads();
    for (int t = threadIdx.x; t < npair * GT_N; t += blockDim.x) {
      int k = t / GT_N, j = t % GT_N;
      int64_t col = col0 + j;
      s_d[t] = col < ndet ? Db[(int64_t)k * ndet + col] : 0.0;
    }
    __syncthreads();
    for (int r0 = 0; r0 < npair; r0 += 16 * 8) {
      double acc[8][4];
#pragma unroll
      for (int i = 0; i < 8; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = 0.0;
      for (int k = 0; k < npair; k++) {
        double dv[4];
#pragma unroll
        for (int j = 0; j < 4; j++) dv[j] = s_d[k * GT_N + tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 8; i++) {
          int r = r0 + ty + 16 * i;
          double gv = r < npair ? s_g[r * npair + k] : 0.0;
#pragma unroll
          for (int j = 0; j < 4; j++) acc[i][j] = fma(gv, dv[j], acc[i][j]);
        }
      }
#pragma unroll
      for (int i = 0; i < 8; i++) {
        int r = r0 + ty + 16 * i;
        if (r >= npair) continue;
#pragma unroll
        for (int j = 0; j < 4; j++) {
          int64_t col = col0 + tx + 16 * j;
          if (col < ndet) Eb[(int64_t)r * ndet + col] = acc[i][j];
        }
      }
    }
  }
}

// sigma(Ia,Ib) = 1/2 sum_P [s_a E_P(Ja,Ib) + s_b E_P(Ia,Jb)] + shift (S^2 c)(Ia,Ib)
// S^2 c = (nsig - ndocc) c - sum over pairs {p,q} with Ia holding one of them
// and Ib the other of s_a s_b c(Ja, Jb)   (S^2 = N_beta - sum E^a_qp E^b_pq)
// E element i: FP64, or (pair_e) the float pair hi + lo written by the
// sliced tensor-core contraction
__device__ __forceinline__ double load_e(const double* __restrict__ Eb, int64_t i, int pair_e) {
  if (!pair_e) return Eb[i];
  const float2 v = reinterpret_cast<const float2*>(Eb)[i];
  return (double)v.x + (double)v.y;
}

// General (not necessarily symmetric) c, alpha table link/masks (nstr
// strings) and beta table linkb/masksb (nstrb strings, the same table for a
// closed shell); S^2 = S-S+ + Ms(Ms+1): diagonal (beta-only orbitals) + msms,
// off-diagonal the alpha-only / beta-only exchanges.
__global__ void k_scatter_fp64(const int32_t* __restrict__ link, const uint32_t* __restrict__ masks,
                               const int32_t* __restrict__ linkb,
                               const uint32_t* __restrict__ masksb, int nstr, int nstrb, int n,
                               int nsigb, double msms, const double* __restrict__ E, int pair_e,
                               const double* __restrict__ c, int64_t c_stride, double shift,
                               const int32_t* __restrict__ active, const int32_t* __restrict__ bmap,
                               double* __restrict__ out, int64_t out_stride) {
  const int bl = blockIdx.y;
  const int b = bmap[bl];
  if (active && !active[b]) return;
  const int npair = n * (n + 1) / 2;
  const int64_t ndet = (int64_t)nstr * nstrb;
  const double* Eb = E + (int64_t)bl * npair * ndet;
  const double* cb = c + (int64_t)b * c_stride;
  double* ob = out + (int64_t)b * out_stride;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ndet;
       i += (int64_t)gridDim.x * blockDim.x) {
    int ia = (int)(i / nstrb), ib = (int)(i % nstrb);
    const int32_t* la = link + (int64_t)ia * npair;
    const int32_t* lb = linkb + (int64_t)ib * npair;
    double acc = 0.0;
    for (int P = 0; P < npair; P++) {
      int32_t ta = la[P], tb = lb[P];
      if (ta >= 0) {
        double x = load_e(Eb, (int64_t)P * ndet + (int64_t)(ta >> 1) * nstrb + ib, pair_e);
        acc += (ta & 1) ? -x : x;
      }
      if (tb >= 0) {
        double x = load_e(Eb, (int64_t)P * ndet + (int64_t)ia * nstrb + (tb >> 1), pair_e);
        acc += (tb & 1) ? -x : x;
      }
    }
    double v = 0.5 * acc;
    if (shift != 0.0) {
      uint32_t ma = masks[ia], mb = masksb[ib];
      double s2 = ((double)(nsigb - __popc(ma & mb)) + msms) * cb[i];
      uint32_t oa = ma & ~mb, ob2 = mb & ~ma;   // open shells of each spin
      for (int q = 0; q < n; q++) {
        if (!((oa >> q) & 1)) continue;
        for (int p = 0; p < n; p++) {
          if (!((ob2 >> p) & 1)) continue;
          int P = p > q ? p * (p + 1) / 2 + q : q * (q + 1) / 2 + p;
          int32_t ta = la[P], tb = lb[P];
          double x = cb[(int64_t)(ta >> 1) * nstrb + (tb >> 1)];
          s2 -= ((ta ^ tb) & 1) ? -x : x;
        }
      }
      v += shift * s2;
    }
    ob[i] = v;
  }
}

// Symmetric c (c(a,b) = c(b,a), the alpha<->beta symmetric Davidson
// vectors): D and E are symmetric in the two strings, so the beta half of
// the scatter is the transpose of the alpha half and
//   sigma = X + X^T + shift S^2 c,  X(a,b) = 1/2 sum_P s_a E_P(J_a, b),
// with every E read coalesced (row J_a, consecutive b).  k_scatter_sym_fp64
// writes X into out; k_finish_sym_fp64 adds the transpose (32 x 32 tile
// pairs in shared memory, in place) and the spin penalty.
__global__ void k_scatter_sym_fp64(const int32_t* __restrict__ link, int nstr, int npair,
                                   const double* __restrict__ E, int pair_e,
                                   const int32_t* __restrict__ active,
                                   const int32_t* __restrict__ bmap, double* __restrict__ out,
                                   int64_t out_stride) {
  const int bl = blockIdx.y;
  const int b = bmap[bl];
  if (active && !active[b]) return;
  const int ndet = nstr * nstr;
  const double* Eb = E + (int64_t)bl * npair * ndet;
  double* ob = out + (int64_t)b * out_stride;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ndet; i += gridDim.x * blockDim.x) {
    const int ia = i / nstr, ib = i - ia * nstr;
    const int32_t* la = link + (int64_t)ia * npair;
    double acc = 0.0;
    for (int P = 0; P < npair; P++) {
      const int32_t ta = la[P];
      if (ta >= 0) {
        const double x = load_e(Eb, (int64_t)P * ndet + (int64_t)(ta >> 1) * nstr + ib, pair_e);
        acc += (ta & 1) ? -x : x;
      }
    }
    ob[i] = 0.5 * acc;
  }
}

__global__ void k_finish_sym_fp64(double* __restrict__ out, int64_t out_stride,
                                  const int32_t* __restrict__ link,
                                  const uint32_t* __restrict__ masks, int nstr, int n, int nsig,
                                  const double* __restrict__ c, int64_t c_stride, double shift,
                                  const int32_t* __restrict__ active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int nt = (nstr + 31) / 32;
  int t = blockIdx.x, I = 0;
  while (t >= nt - I) {
    t -= nt - I;
    I++;
  }
  const int J = I + t;
  __shared__ double sX[2][32][33];
  double* ob = out + (int64_t)b * out_stride;
  const double* cb = c + (int64_t)b * c_stride;
  const int npair = n * (n + 1) / 2;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int h = 0; h < 2; h++) {
    const int r0 = (h ? J : I) * 32, c0 = (h ? I : J) * 32;
    for (int i = ty; i < 32; i += blockDim.x >> 5) {
      const int row = r0 + i, col = c0 + tx;
      sX[h][i][tx] = (row < nstr && col < nstr) ? ob[(int64_t)row * nstr + col] : 0.0;
    }
  }
  __syncthreads();
  // sigma is symmetric: the values of tile (I, J) are formed once and
  // written to both tiles (the transpose through shared memory)
  const int ny = blockDim.x >> 5;
  double v[4];
  for (int k = 0, i = ty; i < 32; i += ny, k++) {
    const int ia = I * 32 + i, ib = J * 32 + tx;
    double s = sX[0][i][tx] + sX[1][tx][i];
    if (shift != 0.0 && ia < nstr && ib < nstr) {
      // evaluated for (min, max): bitwise the same for both elements
      const int lo = min(ia, ib), hi = max(ia, ib);
      const int32_t* la = link + (int64_t)lo * npair;
      const int32_t* lb = link + (int64_t)hi * npair;
      const uint32_t ma = masks[lo], mb = masks[hi];
      double s2 = (double)(nsig - __popc(ma & mb)) * cb[(int64_t)lo * nstr + hi];
      uint32_t oa = ma & ~mb;
      const uint32_t obm = mb & ~ma;
      while (oa) {
        const int q = __ffs(oa) - 1;
        oa &= oa - 1;
        uint32_t o2 = obm;
        while (o2) {
          const int p = __ffs(o2) - 1;
          o2 &= o2 - 1;
          const int P = p > q ? p * (p + 1) / 2 + q : q * (q + 1) / 2 + p;
          const int32_t ta = la[P], tb = lb[P];
          const double x = cb[(int64_t)(ta >> 1) * nstr + (tb >> 1)];
          s2 -= ((ta ^ tb) & 1) ? -x : x;
        }
      }
      s += shift * s2;
    }
    v[k] = s;
  }
  // every read of tile (I, J) and (J, I) went through shared memory above;
  // the CTA owns both tiles, so the in-place stores race with nothing
  for (int k = 0, i = ty; i < 32; i += ny, k++) {
    const int ia = I * 32 + i, ib = J * 32 + tx;
    if (ia < nstr && ib < nstr) ob[(int64_t)ia * nstr + ib] = v[k];
  }
  if (I == J) return;
  __syncthreads();
  for (int k = 0, i = ty; i < 32; i += ny, k++) sX[0][i][tx] = v[k];
  __syncthreads();
  for (int i = ty; i < 32; i += ny) {
    const int ia = J * 32 + i, ib = I * 32 + tx;
    if (ia < nstr && ib < nstr) ob[(int64_t)ia * nstr + ib] = sX[0][tx][i];
  }
}

__global__ void k_s2(const int32_t* __restrict__ link, const uint32_t* __restrict__ masks,
                     const int32_t* __restrict__ linkb, const uint32_t* __restrict__ masksb,
                     int nstr, int nstrb, int n, int nsigb, double msms,
                     const double* __restrict__ c, int64_t c_stride,
                     const int32_t* __restrict__ active, double* __restrict__ out,
                     int64_t out_stride) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int npair = n * (n + 1) / 2;
  const int64_t ndet = (int64_t)nstr * nstrb;
  const double* cb = c + (int64_t)b * c_stride;
  double* ob = out + (int64_t)b * out_stride;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ndet;
       i += (int64_t)gridDim.x * blockDim.x) {
    int ia = (int)(i / nstrb), ib = (int)(i % nstrb);
    const int32_t* la = link + (int64_t)ia * npair;
    const int32_t* lb = linkb + (int64_t)ib * npair;
    uint32_t ma = masks[ia], mb = masksb[ib];
    double s2 = ((double)(nsigb - __popc(ma & mb)) + msms) * cb[i];
    uint32_t oa = ma & ~mb, obm = mb & ~ma;
    for (int q = 0; q < n; q++) {
      if (!((oa >> q) & 1)) continue;
      for (int p = 0; p < n; p++) {
        if (!((obm >> p) & 1)) continue;
        int P = p > q ? p * (p + 1) / 2 + q : q * (q + 1) / 2 + p;
        int32_t ta = la[P], tb = lb[P];
        double x = cb[(int64_t)(ta >> 1) * nstrb + (tb >> 1)];
        s2 -= ((ta ^ tb) & 1) ? -x : x;
      }
    }
    ob[i] = s2;
  }
}

}  // namespace

void sigma_fp64(mbe_ctx* ctx, BinProblem& bp, SigmaWork& w, const double* c, int64_t c_stride,
                double* out, int64_t out_stride, const int32_t* active, double spin_shift,
                bool emulated, bool symmetric) {
  const int npair = bp.npair;
  if (emulated && !w.err.ptr) {
    w.err.reset(&ctx->pool, 1);
    CU_CHECK(cudaMemsetAsync(w.err.ptr, 0, sizeof(int32_t), ctx->stream));
  }
  const int64_t ndet = bp.ndet;
  // sub-batch so that D and E stay within ~2 GB each
  int64_t per = (int64_t)npair * ndet;
  int64_t sb = (int64_t)(2.0e9 / 8.0) / (per > 0 ? per : 1);
  if (sb < 1) sb = 1;
  if (sb > bp.B) sb = bp.B;
  if (w.sub_batch != sb || w.D.n < (size_t)(sb * per)) {
    w.D.reset(&ctx->pool, sb * per);
    w.E.reset(&ctx->pool, sb * per);
    w.sub_batch = sb;
  }
  std::vector<int32_t> bm(bp.B);
  for (int i = 0; i < bp.B; i++) bm[i] = i;
  DevBuf<int32_t> bmap(&ctx->pool, bp.B);
  CU_CHECK(cudaMemcpyAsync(bmap.ptr, bm.data(), sizeof(int32_t) * bp.B, cudaMemcpyHostToDevice,
                           ctx->stream));
  for (int64_t b0 = 0; b0 < bp.B; b0 += sb) {
    const int nb = (int)std::min<int64_t>(sb, bp.B - b0);
    sigma_fp64_raw(ctx, bp.n, bp.nsig, bp.nstr, bp.tab->link.ptr, bp.tab->masks.ptr, bp.gp.ptr, c,
                   c_stride, out, out_stride, active, bmap.ptr + b0, nb, w.D.ptr, w.E.ptr,
                   spin_shift, emulated, w.err.ptr, symmetric && bp.closed(), (int)b0, bp.nsigb,
                   bp.nstrb, bp.tabb->link.ptr, bp.tabb->masks.ptr);
  }
}

void sigma_fp64_raw(mbe_ctx* ctx, int n, int nsig, int nstr, const int32_t* link,
                    const uint32_t* masks, const double* gp, const double* c, int64_t c_stride,
                    double* out, int64_t out_stride, const int32_t* active, const int32_t* bmap,
                    int nb, double* D, double* E, double spin_shift, bool emulated, int32_t* err,
                    bool symmetric, int b_first, int nsigb, int nstrb, const int32_t* linkb,
                    const uint32_t* masksb) {
  if (nsigb < 0) {   // closed shell: beta strings = alpha strings
    nsigb = nsig;
    nstrb = nstr;
    linkb = link;
    masksb = masks;
  }
  const double msms = 0.25 * (nsig - nsigb) * (nsig - nsigb + 2);   // Ms(Ms+1)
  const int npair = n * (n + 1) / 2;
  const int64_t ndet = (int64_t)nstr * nstrb;
  int64_t blocks = (ndet + 255) / 256;
  if (blocks > 2048) blocks = 2048;
  const size_t smem_c = sizeof(double) * (npair * npair + npair * GT_N);
  static bool attr_set[MBE_MAX_DEVICES] = {false};
  once_per_device(attr_set, ctx->device, [] {
    CU_CHECK(cudaFuncSetAttribute(k_contract_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  200 * 1024));
  });
  int64_t cblocks = (ndet + GT_N - 1) / GT_N;
  if (cblocks > 1024) cblocks = 1024;
  const dim3 g1((unsigned)blocks, nb);
  k_gather_fp64<<<g1, 256, 0, ctx->stream>>>(link, linkb, nstr, nstrb, npair, c, c_stride, active,
                                              bmap, D);
  CU_LAUNCH_CHECK();
  cudaEvent_t ev;
  ctx->fp64_timer.begin(ctx->stream, ctx->opt.timing != 0, &ev);
  if (emulated) {
    contract_ozaki(ctx, gp, npair, D, ndet, nb, active, bmap, E, err);
  } else {
    k_contract_fp64<<<dim3((unsigned)cblocks, nb), 256, smem_c, ctx->stream>>>(gp, npair, D, ndet,
                                                                             active, bmap, E);
    CU_LAUNCH_CHECK();
  }
  ctx->fp64_timer.end(ctx->stream, ev);
  ctx->stats.fp64_launches += 1;
  if (symmetric) {
    k_scatter_sym_fp64<<<g1, 256, 0, ctx->stream>>>(link, nstr, npair, E, emulated ? 1 : 0,
                                                    active, bmap, out, out_stride);
    CU_LAUNCH_CHECK();
    // the sub-batch is the contiguous tuple range [b_first, b_first + nb)
    const int ntl = (nstr + 31) / 32;
    const int b0 = b_first;
    k_finish_sym_fp64<<<dim3((unsigned)(ntl * (ntl + 1) / 2), nb), 256, 0, ctx->stream>>>(
        out + (int64_t)b0 * out_stride, out_stride, link, masks, nstr, n, nsig,
        c + (int64_t)b0 * c_stride, c_stride, spin_shift, active ? active + b0 : nullptr);
    CU_LAUNCH_CHECK();
  } else {
    k_scatter_fp64<<<g1, 256, 0, ctx->stream>>>(link, masks, linkb, masksb, nstr, nstrb, n, nsigb,
                                                msms, E, emulated ? 1 : 0, c, c_stride,
                                                spin_shift, active, bmap, out, out_stride);
    CU_LAUNCH_CHECK();
  }
}

void s2_apply(mbe_ctx* ctx, BinProblem& bp, const double* c, int64_t c_stride, double* out,
              int64_t out_stride, const int32_t* active) {
  int64_t blocks = (bp.ndet + 255) / 256;
  if (blocks > 2048) blocks = 2048;
  dim3 g((unsigned)blocks, bp.B);
  k_s2<<<g, 256, 0, ctx->stream>>>(bp.tab->link.ptr, bp.tab->masks.ptr, bp.tabb->link.ptr,
                                   bp.tabb->masks.ptr, bp.nstr, bp.nstrb, bp.n, bp.nsigb,
                                   bp.msms(), c, c_stride, active, out, out_stride);
  CU_LAUNCH_CHECK();
}

// ------------------------------------------------------------ warm starts
namespace {

__global__ void k_f64_to_f32(const double* __restrict__ src, float* __restrict__ dst, int64_t n) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    dst[k] = (float)src[k];
}

// V[b][0] of the child tuple from the parent's vector: every parent string
// (n - 1 orbitals) gains the added orbital at active position jo -- empty,
// or occupied in both strings, which moves its creation operators past the
// electrons below it: sign (-1)^(n_alpha below + n_beta below).  The child
// row is zeroed first by k_zero_start.
template <typename T>
__global__ void k_zero_start(const int32_t* __restrict__ bidx, int64_t N, T* __restrict__ V,
                             int64_t vstride) {
  T* Vb = V + (int64_t)bidx[blockIdx.y] * vstride;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * blockDim.x)
    Vb[k] = (T)0;
}

template <typename T>
__global__ void k_parent_guess(const float* const* __restrict__ src,
                               const int32_t* __restrict__ bidx, const int32_t* __restrict__ jo,
                               const int32_t* __restrict__ occ,
                               const uint32_t* __restrict__ masks_v, int nstr_v,
                               const uint32_t* __restrict__ masks_o, int nstr_o, int nstr,
                               T* __restrict__ V, int64_t vstride) {
  const int e = blockIdx.y;
  const int o = occ[e], j = jo[e];
  const uint32_t* pm = o ? masks_o : masks_v;
  const int np = o ? nstr_o : nstr_v;
  const int64_t Np = (int64_t)np * np;
  const uint32_t low = (1u << j) - 1u;
  const float* sv = src[e];
  T* Vb = V + (int64_t)bidx[e] * vstride;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Np;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int ia = (int)(i / np), ib = (int)(i - (int64_t)ia * np);
    const uint32_t ma = pm[ia], mb = pm[ib];
    const uint32_t ca = (ma & low) | ((ma & ~low) << 1) | ((uint32_t)o << j);
    const uint32_t cb = (mb & low) | ((mb & ~low) << 1) | ((uint32_t)o << j);
    const int neg = o ? ((__popc(ma & low) + __popc(mb & low)) & 1) : 0;
    const float v = sv[i];
    Vb[(int64_t)mask_rank(ca) * nstr + mask_rank(cb)] = (T)(neg ? -v : v);
  }
}

// the inserted vectors are FP32 copies: normalise each in FP64 (the
// Rayleigh-Ritz step assumes an orthonormal basis), one block per tuple
template <typename T>
__global__ void k_normalize_start(const int32_t* __restrict__ bidx, int64_t N, T* __restrict__ V,
                                  int64_t vstride) {
  T* Vb = V + (int64_t)bidx[blockIdx.x] * vstride;
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t k = threadIdx.x; k < N; k += blockDim.x) s += (double)Vb[k] * (double)Vb[k];
  for (int off = 16; off; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  __shared__ double inv;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
    inv = t > 0.0 ? 1.0 / sqrt(t) : 1.0;
  }
  __syncthreads();
  for (int64_t k = threadIdx.x; k < N; k += blockDim.x) Vb[k] = (T)((double)Vb[k] * inv);
}

}  // namespace

void launch_parent_guess(mbe_ctx* ctx, const GuessPlan& plan, int n, int nsig, int nstr,
                         float* V32, double* V64, int64_t vstride) {
  const int ne = (int)plan.b.size();
  if (ne == 0 || n < 2) return;
  bool any_o = false, any_v = false;
  for (int e = 0; e < ne; e++) (plan.occ[e] ? any_o : any_v) = true;
  const StringTables* tv = any_v ? get_tables(ctx, n - 1, nsig) : nullptr;
  const StringTables* to = (any_o && nsig >= 1) ? get_tables(ctx, n - 1, nsig - 1) : nullptr;
  if (any_o && !to) throw MbeError{MBE_ESTATE, "occupied added orbital without electrons"};
  DevBuf<int32_t> bidx(&ctx->pool, ne), jo(&ctx->pool, ne), occ(&ctx->pool, ne);
  DevBuf<const float*> src(&ctx->pool, ne);
  cudaStream_t st = ctx->stream;
  CU_CHECK(cudaMemcpyAsync(bidx.ptr, plan.b.data(), sizeof(int32_t) * ne, cudaMemcpyHostToDevice, st));
  CU_CHECK(cudaMemcpyAsync(jo.ptr, plan.jo.data(), sizeof(int32_t) * ne, cudaMemcpyHostToDevice, st));
  CU_CHECK(cudaMemcpyAsync(occ.ptr, plan.occ.data(), sizeof(int32_t) * ne, cudaMemcpyHostToDevice, st));
  CU_CHECK(cudaMemcpyAsync(src.ptr, plan.src.data(), sizeof(const float*) * ne,
                           cudaMemcpyHostToDevice, st));
  const int64_t N = (int64_t)nstr * nstr;
  const dim3 g((unsigned)std::min<int64_t>((N + 255) / 256, 1024), ne);
  const uint32_t* mv = tv ? tv->masks.ptr : nullptr;
  const uint32_t* mo = to ? to->masks.ptr : nullptr;
  const int nv = tv ? tv->nstr : 0, no = to ? to->nstr : 0;
  if (V32) {
    k_zero_start<float><<<g, 256, 0, st>>>(bidx.ptr, N, V32, vstride);
    CU_LAUNCH_CHECK();
    k_parent_guess<float><<<g, 256, 0, st>>>(src.ptr, bidx.ptr, jo.ptr, occ.ptr, mv, nv, mo, no,
                                             nstr, V32, vstride);
    CU_LAUNCH_CHECK();
    k_normalize_start<float><<<ne, 1024, 0, st>>>(bidx.ptr, N, V32, vstride);
  } else {
    k_zero_start<double><<<g, 256, 0, st>>>(bidx.ptr, N, V64, vstride);
    CU_LAUNCH_CHECK();
    k_parent_guess<double><<<g, 256, 0, st>>>(src.ptr, bidx.ptr, jo.ptr, occ.ptr, mv, nv, mo, no,
                                              nstr, V64, vstride);
    CU_LAUNCH_CHECK();
    k_normalize_start<double><<<ne, 1024, 0, st>>>(bidx.ptr, N, V64, vstride);
  }
  CU_LAUNCH_CHECK();
}

void convert_f64_to_f32(mbe_ctx* ctx, const double* src, float* dst, int64_t n) {
  if (n <= 0) return;
  k_f64_to_f32<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, ctx->stream>>>(
      src, dst, n);
  CU_LAUNCH_CHECK();
}

void launch_finish_sym_fp64(mbe_ctx* ctx, const BinProblem& bp, double* out, int64_t out_stride,
                            const double* c, int64_t c_stride, double spin_shift,
                            const int32_t* active) {
  const int ntl = (bp.nstr + 31) / 32;
  k_finish_sym_fp64<<<dim3((unsigned)(ntl * (ntl + 1) / 2), bp.B), 256, 0, ctx->stream>>>(
      out, out_stride, bp.tab->link.ptr, bp.tab->masks.ptr, bp.nstr, bp.n, bp.nsig, c, c_stride,
      spin_shift, active);
  CU_LAUNCH_CHECK();
}
