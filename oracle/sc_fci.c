/*
 * Oracle (test infrastructure only): determinant-driven configuration
 * interaction in the FULL orbital space by the Slater-Condon rules.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference leg may load this library.  It shares no code with the CUDA
 * path: no effective integrals, no string link tables, no pair-packed
 * sigma; every matrix element is evaluated from the full-space h_pq and
 * (pq|rs) on full-space spin-orbital determinants, so the frozen-core fold
 * of a CASCI (Sec. 2, Fig. 2: occupied orbitals outside the active space are
 * inactive, virtuals outside it are deleted) is exercised implicitly.
 *
 * Conventions
 *   A determinant is a^+_{alpha string} a^+_{beta string} |0>, creation
 *   operators in ascending spin-orbital order with all alpha spin-orbitals
 *   before all beta ones.  Spin-orbital k: alpha orbital p -> k = p,
 *   beta orbital p -> k = 128 + p (norb <= 128).  Every fermionic sign is
 *   obtained by applying the operators one at a time, each contributing
 *   (-1)^(number of occupied spin-orbitals below it).
 *   Strings are passed as pairs of uint64 (lo, hi) orbital bit masks and
 *   must be sorted ascending by (hi, lo).  Determinant index = ia*nb + ib.
 *   ERIs are chemists' (pq|rs), packed 4-fold as an npair x npair matrix.
 *
 * Hamiltonian: H = sum h_pq a+_p a_q + 1/2 sum (pq|rs) a+_p a+_r a_s a_q
 * (spin-orbital sums with spin deltas), Slater-Condon rules (textbook, e.g.
 * Szabo & Ostlund, Sec. 2.3):
 *   <I|H|I>  = sum_k h_kk + 1/2 sum_{k,l} [(kk|ll) - d(s_k,s_l)(kl|lk)]
 *   single i->a:  sign * [h_ai + sum_{k in I, k != i} ((ai|kk) - d(s_a,s_k)(ak|ki))]
 *   double ij->ab: sign * [<ab|ij> - <ab|ji>],  <ab|ij> = d d (ai|bj)
 * with sign from a+_a a+_b a_j a_i |I> (resp. a+_a a_i |I>).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { uint64_t w[4]; } sdet;

static inline int sbit(const sdet *d, int k) { return (int)((d->w[k >> 6] >> (k & 63)) & 1ULL); }

static inline int nbelow(const sdet *d, int k) {
    int c = 0, wi = k >> 6;
    for (int i = 0; i < wi; i++) c += __builtin_popcountll(d->w[i]);
    if (k & 63) c += __builtin_popcountll(d->w[wi] & ((1ULL << (k & 63)) - 1ULL));
    return c;
}

/* a_k |d>: returns the sign, or 0 if k is empty. */
static inline int op_ann(sdet *d, int k) {
    if (!sbit(d, k)) return 0;
    int s = (nbelow(d, k) & 1) ? -1 : 1;
    d->w[k >> 6] &= ~(1ULL << (k & 63));
    return s;
}

/* a^+_k |d>: returns the sign, or 0 if k is occupied. */
static inline int op_cre(sdet *d, int k) {
    if (sbit(d, k)) return 0;
    int s = (nbelow(d, k) & 1) ? -1 : 1;
    d->w[k >> 6] |= (1ULL << (k & 63));
    return s;
}

static inline long pidx(int p, int q) { return p >= q ? (long)p * (p + 1) / 2 + q : (long)q * (q + 1) / 2 + p; }

typedef struct {
    int norb; long npair;
    const double *h, *eri;
} ints_t;

static inline double ERI(const ints_t *I, int p, int q, int r, int s) {
    return I->eri[pidx(p, q) * I->npair + pidx(r, s)];
}

/* binary search of a (lo, hi) string in a list sorted by (hi, lo). */
static long find_str(const uint64_t *strs, long n, uint64_t lo, uint64_t hi) {
    long a = 0, b = n - 1;
    while (a <= b) {
        long m = (a + b) >> 1;
        uint64_t mlo = strs[2 * m], mhi = strs[2 * m + 1];
        if (mhi == hi && mlo == lo) return m;
        if (mhi < hi || (mhi == hi && mlo < lo)) a = m + 1; else b = m - 1;
    }
    return -1;
}

static inline sdet make_det(const uint64_t *a, const uint64_t *b) {
    sdet d; d.w[0] = a[0]; d.w[1] = a[1]; d.w[2] = b[0]; d.w[3] = b[1]; return d;
}

static inline long det_index(const sdet *d, const uint64_t *astr, long na, const uint64_t *bstr, long nb) {
    long ia = find_str(astr, na, d->w[0], d->w[1]);
    if (ia < 0) return -1;
    long ib = find_str(bstr, nb, d->w[2], d->w[3]);
    if (ib < 0) return -1;
    return ia * nb + ib;
}

static int occ_list(const sdet *d, int norb, int *occ) {
    int n = 0;
    for (int s = 0; s < 2; s++)
        for (int p = 0; p < norb; p++) if (sbit(d, 128 * s + p)) occ[n++] = 128 * s + p;
    return n;
}

static double diag_elem(const ints_t *I, const sdet *d) {
    int occ[256]; int n = occ_list(d, I->norb, occ);
    double e = 0.0;
    for (int x = 0; x < n; x++) {
        int k = occ[x] & 127;
        e += I->h[k * I->norb + k];
    }
    double e2 = 0.0;
    for (int x = 0; x < n; x++)
        for (int y = 0; y < n; y++) {
            int k = occ[x] & 127, l = occ[y] & 127;
            e2 += ERI(I, k, k, l, l);
            if ((occ[x] >> 7) == (occ[y] >> 7)) e2 -= ERI(I, k, l, l, k);
        }
    return e + 0.5 * e2;
}

/* <J|H|I> for J = a+_a a_i I (same spin), without the sign. */
static double single_elem(const ints_t *I, const sdet *ket, int i, int a) {
    int occ[256]; int n = occ_list(ket, I->norb, occ);
    int oi = i & 127, oa = a & 127, si = i >> 7;
    double e = I->h[oa * I->norb + oi];
    for (int x = 0; x < n; x++) {
        if (occ[x] == i) continue;
        int k = occ[x] & 127;
        e += ERI(I, oa, oi, k, k);
        if ((occ[x] >> 7) == si) e -= ERI(I, oa, k, k, oi);
    }
    return e;
}

/* <ab|ij> - <ab|ji> for spin-orbitals (physicists' notation). */
static double double_elem(const ints_t *I, int i, int j, int a, int b) {
    double e = 0.0;
    if ((a >> 7) == (i >> 7) && (b >> 7) == (j >> 7)) e += ERI(I, a & 127, i & 127, b & 127, j & 127);
    if ((a >> 7) == (j >> 7) && (b >> 7) == (i >> 7)) e -= ERI(I, a & 127, j & 127, b & 127, i & 127);
    return e;
}

typedef struct {
    const ints_t *I;
    long na, nb;
    const uint64_t *astr, *bstr;
    int nspace;          /* spin-orbitals that may change occupation */
    int space[256];
} space_t;

/* Visit every determinant J != I connected to I by a single or double
 * excitation within the space; call f(J index, <J|H|I>). */
typedef void (*visit_fn)(void *ctx, long j, double hji);

static void for_each_connected(const space_t *S, const sdet *ket, visit_fn f, void *ctx) {
    int holes[256], parts[256], nh = 0, np = 0;
    for (int x = 0; x < S->nspace; x++) {
        int k = S->space[x];
        if (sbit(ket, k)) holes[nh++] = k; else parts[np++] = k;
    }
    /* singles */
    for (int x = 0; x < nh; x++)
        for (int y = 0; y < np; y++) {
            int i = holes[x], a = parts[y];
            if ((i >> 7) != (a >> 7)) continue;
            sdet d = *ket;
            int sg = op_ann(&d, i); sg *= op_cre(&d, a);
            long j = det_index(&d, S->astr, S->na, S->bstr, S->nb);
            if (j < 0) continue;
            f(ctx, j, sg * single_elem(S->I, ket, i, a));
        }
    /* doubles: i < j holes, a < b particles, spin conserved */
    for (int x = 0; x < nh; x++)
        for (int x2 = x + 1; x2 < nh; x2++)
            for (int y = 0; y < np; y++)
                for (int y2 = y + 1; y2 < np; y2++) {
                    int i = holes[x], jj = holes[x2], a = parts[y], b = parts[y2];
                    int ms_h = (i >> 7) + (jj >> 7), ms_p = (a >> 7) + (b >> 7);
                    if (ms_h != ms_p) continue;
                    sdet d = *ket;
                    int sg = op_ann(&d, i);
                    sg *= op_ann(&d, jj);
                    sg *= op_cre(&d, b);
                    sg *= op_cre(&d, a);
                    long j = det_index(&d, S->astr, S->na, S->bstr, S->nb);
                    if (j < 0) continue;
                    double v = double_elem(S->I, i, jj, a, b);
                    if (v != 0.0) f(ctx, j, sg * v);
                }
}

static void setup_space(space_t *S, const ints_t *I, long na, const uint64_t *astr, long nb, const uint64_t *bstr) {
    S->I = I; S->na = na; S->nb = nb; S->astr = astr; S->bstr = bstr;
    /* orbitals whose occupation varies across the string list */
    uint64_t orA[2] = {0, 0}, andA[2] = {~0ULL, ~0ULL}, orB[2] = {0, 0}, andB[2] = {~0ULL, ~0ULL};
    for (long x = 0; x < na; x++) for (int w = 0; w < 2; w++) { orA[w] |= astr[2 * x + w]; andA[w] &= astr[2 * x + w]; }
    for (long x = 0; x < nb; x++) for (int w = 0; w < 2; w++) { orB[w] |= bstr[2 * x + w]; andB[w] &= bstr[2 * x + w]; }
    S->nspace = 0;
    for (int p = 0; p < I->norb; p++) {
        uint64_t m = 1ULL << (p & 63); int w = p >> 6;
        if ((orA[w] & m) && !(andA[w] & m)) S->space[S->nspace++] = p;
    }
    for (int p = 0; p < I->norb; p++) {
        uint64_t m = 1ULL << (p & 63); int w = p >> 6;
        if ((orB[w] & m) && !(andB[w] & m)) S->space[S->nspace++] = 128 + p;
    }
}

/* ---------------- exported entry points ---------------- */

void oracle_hdiag(int norb, const double *h, const double *eri,
                  long na, const uint64_t *astr, long nb, const uint64_t *bstr, double *out) {
    ints_t I = {norb, (long)norb * (norb + 1) / 2, h, eri};
    #pragma omp parallel for schedule(dynamic, 16)
    for (long ia = 0; ia < na; ia++)
        for (long ib = 0; ib < nb; ib++) {
            sdet d = make_det(astr + 2 * ia, bstr + 2 * ib);
            out[ia * nb + ib] = diag_elem(&I, &d);
        }
}

typedef struct { const double *c; double acc; } sig_ctx;
static void sig_visit(void *ctx, long j, double hji) { sig_ctx *s = (sig_ctx *)ctx; s->acc += hji * s->c[j]; }

/* sigma_I = sum_J <I|H|J> c_J  (pull form; <I|H|J> = <J|H|I>). */
void oracle_sigma(int norb, const double *h, const double *eri,
                  long na, const uint64_t *astr, long nb, const uint64_t *bstr,
                  const double *c, double *sigma) {
    ints_t I = {norb, (long)norb * (norb + 1) / 2, h, eri};
    space_t S; setup_space(&S, &I, na, astr, nb, bstr);
    #pragma omp parallel for schedule(dynamic, 4)
    for (long ia = 0; ia < na; ia++)
        for (long ib = 0; ib < nb; ib++) {
            sdet d = make_det(astr + 2 * ia, bstr + 2 * ib);
            sig_ctx sc = {c, 0.0};
            for_each_connected(&S, &d, sig_visit, &sc);
            long i = ia * nb + ib;
            sigma[i] = sc.acc + diag_elem(&I, &d) * c[i];
        }
}

/* sigma_I for the listed determinants only: out[x] = sum_J <I|H|J> c_J with
 * I = rows[x] (the loop of oracle_sigma restricted to those rows). */
void oracle_sigma_rows(int norb, const double *h, const double *eri,
                       long na, const uint64_t *astr, long nb, const uint64_t *bstr,
                       const double *c, long nrows, const long *rows, double *out) {
    ints_t I = {norb, (long)norb * (norb + 1) / 2, h, eri};
    space_t S; setup_space(&S, &I, na, astr, nb, bstr);
    #pragma omp parallel for schedule(dynamic, 4)
    for (long x = 0; x < nrows; x++) {
        long i = rows[x];
        sdet d = make_det(astr + 2 * (i / nb), bstr + 2 * (i % nb));
        sig_ctx sc = {c, 0.0};
        for_each_connected(&S, &d, sig_visit, &sc);
        out[x] = sc.acc + diag_elem(&I, &d) * c[i];
    }
}

typedef struct { double *row; } row_ctx;
static void row_visit(void *ctx, long j, double hji) { ((row_ctx *)ctx)->row[j] += hji; }

/* Dense H (ndet x ndet, row-major); row I holds <J|H|I> evaluated with I as ket. */
void oracle_hdense(int norb, const double *h, const double *eri,
                   long na, const uint64_t *astr, long nb, const uint64_t *bstr, double *H) {
    ints_t I = {norb, (long)norb * (norb + 1) / 2, h, eri};
    space_t S; setup_space(&S, &I, na, astr, nb, bstr);
    long nd = na * nb;
    #pragma omp parallel for schedule(dynamic, 4)
    for (long i = 0; i < nd; i++) {
        double *row = H + i * nd;
        memset(row, 0, sizeof(double) * nd);
        sdet d = make_det(astr + 2 * (i / nb), bstr + 2 * (i % nb));
        row_ctx rc = {row};
        for_each_connected(&S, &d, row_visit, &rc);
        row[i] += diag_elem(&I, &d);
    }
}

/* Spin-summed full-space 1- and 2-RDMs of the normalised vector c:
 *   rdm1[p,q]      = sum_s <a+_ps a_qs>
 *   rdm2[p,q,r,s]  = sum_{s1,s2} <a+_{p s1} a+_{r s2} a_{s s2} a_{q s1}>
 * (so E = sum h_pq rdm1_pq + 1/2 sum (pq|rs) rdm2_pqrs).  Operators are
 * applied to each ket one at a time; a result outside the determinant list
 * has zero overlap with c and is skipped. */
void oracle_rdm12(int norb, long na, const uint64_t *astr, long nb, const uint64_t *bstr,
                  const double *c, double *rdm1, double *rdm2) {
    long n2 = (long)norb * norb, n4 = n2 * n2;
    memset(rdm1, 0, sizeof(double) * n2);
    memset(rdm2, 0, sizeof(double) * n4);
    /* spin-orbitals that occur in some determinant */
    uint64_t orA[2] = {0, 0}, orB[2] = {0, 0};
    for (long x = 0; x < na; x++) for (int w = 0; w < 2; w++) orA[w] |= astr[2 * x + w];
    for (long x = 0; x < nb; x++) for (int w = 0; w < 2; w++) orB[w] |= bstr[2 * x + w];
    int allowed[256], nal = 0;
    for (int p = 0; p < norb; p++) if (orA[p >> 6] >> (p & 63) & 1ULL) allowed[nal++] = p;
    for (int p = 0; p < norb; p++) if (orB[p >> 6] >> (p & 63) & 1ULL) allowed[nal++] = 128 + p;
    long nd = na * nb;
    #pragma omp parallel
    {
        double *g1 = (double *)calloc(n2, sizeof(double));
        double *g2 = (double *)calloc(n4, sizeof(double));
        #pragma omp for schedule(dynamic, 8)
        for (long jx = 0; jx < nd; jx++) {
            double cj = c[jx];
            if (cj == 0.0) continue;
            sdet ket = make_det(astr + 2 * (jx / nb), bstr + 2 * (jx % nb));
            for (int xq = 0; xq < nal; xq++) {
                int Q = allowed[xq];
                sdet d1 = ket; int s1 = op_ann(&d1, Q);
                if (!s1) continue;
                /* one-body: a+_P a_Q */
                for (int xp = 0; xp < nal; xp++) {
                    int P = allowed[xp];
                    if ((P >> 7) != (Q >> 7)) continue;
                    sdet d = d1; int s = op_cre(&d, P);
                    if (!s) continue;
                    long k = det_index(&d, astr, na, bstr, nb);
                    if (k < 0) continue;
                    g1[(P & 127) * norb + (Q & 127)] += c[k] * s1 * s * cj;
                }
                /* two-body: a+_P a+_R a_S a_Q */
                for (int xs = 0; xs < nal; xs++) {
                    int Sx = allowed[xs];
                    sdet d2 = d1; int s2 = op_ann(&d2, Sx);
                    if (!s2) continue;
                    for (int xr = 0; xr < nal; xr++) {
                        int R = allowed[xr];
                        if ((R >> 7) != (Sx >> 7)) continue;
                        sdet d3 = d2; int s3 = op_cre(&d3, R);
                        if (!s3) continue;
                        for (int xp = 0; xp < nal; xp++) {
                            int P = allowed[xp];
                            if ((P >> 7) != (Q >> 7)) continue;
                            sdet d4 = d3; int s4 = op_cre(&d4, P);
                            if (!s4) continue;
                            long k = det_index(&d4, astr, na, bstr, nb);
                            if (k < 0) continue;
                            long idx = (((long)(P & 127) * norb + (Q & 127)) * norb + (R & 127)) * norb + (Sx & 127);
                            g2[idx] += c[k] * s1 * s2 * s3 * s4 * cj;
                        }
                    }
                }
            }
        }
        #pragma omp critical
        {
            for (long x = 0; x < n2; x++) rdm1[x] += g1[x];
            for (long x = 0; x < n4; x++) rdm2[x] += g2[x];
        }
        free(g1); free(g2);
    }
}

/* (S^2 c)_I for an Ms = 0 vector, with S^2 = S- S+ (valid for Ms = 0),
 * S+ = sum_q a+_{q alpha} a_{q beta}, S- = sum_p a+_{p beta} a_{p alpha}.
 * Pull form: S^2 is real symmetric, so (S^2 c)_I = sum_K <K|S^2|I> c_K with
 * K = a+_{p beta} a_{p alpha} a+_{q alpha} a_{q beta} |I> built one operator
 * at a time.  diag_out (optional) receives <I|S^2|I>. */
void oracle_s2(int norb, long na, const uint64_t *astr, long nb, const uint64_t *bstr,
               const double *c, double *out, double *diag_out) {
    long nd = na * nb;
    #pragma omp parallel for schedule(dynamic, 8)
    for (long i = 0; i < nd; i++) {
        sdet ket = make_det(astr + 2 * (i / nb), bstr + 2 * (i % nb));
        double acc = 0.0, dg = 0.0;
        for (int q = 0; q < norb; q++) {
            sdet d1 = ket; int s1 = op_ann(&d1, 128 + q);
            if (!s1) continue;
            int s2 = op_cre(&d1, q);
            if (!s2) continue;
            for (int p = 0; p < norb; p++) {
                sdet d2 = d1; int s3 = op_ann(&d2, p);
                if (!s3) continue;
                int s4 = op_cre(&d2, 128 + p);
                if (!s4) continue;
                long k = det_index(&d2, astr, na, bstr, nb);
                if (k < 0) continue;
                double v = (double)(s1 * s2 * s3 * s4);
                if (c) acc += v * c[k];
                if (k == i) dg += v;
            }
        }
        if (out) out[i] = acc;
        if (diag_out) diag_out[i] = dg;
    }
}
