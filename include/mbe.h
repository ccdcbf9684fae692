/*
 * mbe.h -- C ABI of the GB300 MBE-FCI hot path.
 *
 * Many-body expanded full configuration interaction with a (multi-
 * determinantal) CAS expansion reference, Eriksen & Gauss, "Many-Body
 * Expanded Full Configuration Interaction. II. Strongly Correlated Regime"
 * (arXiv:1905.02786), Sec. 2:
 *   Eq. 1  E = sum over orders of the increments,
 *   Eq. 2  increment of a tuple = its CASCI energy minus those of all proper
 *          subtuples (S_m = unique subtuples of length m),
 *   Eq. 3  the same with a reference space Pi: every CASCI correlates Pi plus
 *          the tuple; the order-0 term is the CASCI energy of Pi,
 *   Fig. 2 occupied orbitals outside Pi+tuple are inactive (doubly
 *          occupied), virtuals outside it are deleted.
 *
 * Every CASCI is solved on the GPU by a Davidson iteration on a
 * string-driven sigma vector; increments are assembled through a device
 * hash of tuples and screened; the energy gradient is assembled from the
 * tuples' RDMs (Hellmann-Feynman).
 *
 * General conventions
 *  - Return value: MBE_OK (0) or a negative MBE_E* code; the message of the
 *    last failure of a context is returned by mbe_last_error().
 *  - Ownership: every array argument is caller-owned HOST memory unless the
 *    name ends in _dev (caller-owned DEVICE memory on the context's device).
 *    Inputs are copied before the call returns; the library never keeps a
 *    caller pointer.
 *  - Threads: a context is not thread-safe; use one context per host thread.
 *  - Orbitals are 0-based; orbitals 0 .. nelec/2-1 are the occupied ones of
 *    the closed-shell (RHF-like) reference determinant.  norb <= 128.
 *  - Integrals are real: h is norb x norb row-major (symmetric); the
 *    two-electron integrals (pq|rs) (chemists' notation, 8-fold symmetric)
 *    are passed packed 4-fold as a symmetric npair x npair row-major matrix
 *    eri[P*npair + Q], npair = norb(norb+1)/2, P = p(p+1)/2 + q for p >= q.
 *  - Energies are total electronic energies in Eh (the paper's correlation
 *    energies differ by a constant, which affects only the order-0 term).
 *  - State: the lowest singlet (S = 0, Ms = 0) of each CASCI.
 */
#ifndef MBE_H
#define MBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  MBE_OK = 0,
  MBE_EINVAL = -1,    /* bad argument (size, index, NaN/Inf input, order)   */
  MBE_ENOMEM = -2,    /* device allocation failed or memory cap exceeded    */
  MBE_ECUDA = -3,     /* a CUDA runtime call failed                          */
  MBE_ENOCONV = -4,   /* some CASCI did not converge (see status_out)       */
  MBE_ELOOKUP = -5,   /* a subtuple increment was missing from the hash     */
  MBE_ESTATE = -6,    /* call out of sequence (e.g. no integrals loaded)    */
  MBE_ETIMEOUT = -7   /* a bounded device-side wait gave up (opt.wait_limit);
                         the kernel returned, the context stays usable      */
};

/* Precision of the sigma-vector contraction. */
enum {
  MBE_FP64 = 0,          /* every step in FP64 (CUDA-core FP64 contraction)  */
  MBE_MIXED_BF16X3 = 1,  /* Davidson vectors in FP32; their sigma vectors as
                            split-BF16x3 on tcgen05 tensor cores with FP32
                            accumulation; refinement rounds ("exact points")
                            with FP64-grade sigma vectors, the Rayleigh
                            quotient and residual formed with error-free
                            FP32 products and sums; the Ritz step is an FP32
                            Jacobi eigensolver refined by FP64 Newton steps,
                            Gram-Schmidt runs in FP32 with FP64 sums across
                            threads, the energy, <S^2> and the increment
                            sums are FP64                                    */
  MBE_EMULATED_FP64 = 2  /* every sigma vector with the (kl|ij) contraction
                            emulated to ~1e-10 relative on tcgen05 tensor
                            cores (exact 8-bit slices, grouped FP32
                            accumulators, FP64 recombination)                */
};

typedef struct mbe_options {
  int precision;        /* MBE_FP64 or MBE_MIXED_BF16X3                      */
  int max_batch;        /* max tuples solved together in one bin (>= 1); 1
                           gives the one-tuple-at-a-time path               */
  int max_subspace;     /* Davidson subspace size before restart (4..32); in
                           the mixed mode a refinement round that fills its
                           subspace makes the later rounds of the batch use
                           up to 12 more vectors (at most 32)               */
  int max_iter;         /* Davidson iteration cap per tuple                  */
  double conv_tol_r;    /* residual-norm tolerance of the Davidson iteration */
  double conv_tol_e;    /* energy-change tolerance                           */
  double spin_shift;    /* lambda of H + lambda S^2 (lifts S >= 2 states)    */
  int keep_ci;          /* keep, on the device, the packed active-space RDMs
                           of every converged CASCI for the energy backward
                           (formed from the vector right after its batch
                           converges; the vector itself is not kept)       */
  int deterministic;    /* 1: fixed-order reductions only (no float atomics) */
  int64_t mem_cap_bytes;/* cap on device memory the context may allocate; 0 =
                           no cap (exceeding it returns MBE_ENOMEM)          */
  int timing;           /* 1: time the sigma contraction launches with CUDA
                           events (mbe_stats.dom_ms)                         */
  int verbose;          /* 1: print per-iteration Davidson residual summaries
                           to stderr                                         */
  int backward_share;   /* what mbe_energy_backward sums: 0 the whole
                           expansion (every RDM set must be held here);
                           1 only the tuples whose RDMs this context
                           holds (tuples sharded over contexts); 2 as 1 plus
                           the reference-space term (exactly one context of
                           a sharded run)                                    */
  int warm_start;       /* 1: a tuple starts its Davidson iteration from the
                           converged vector of a parent (the tuple less one
                           orbital, solved at the previous order) with the
                           orbital added; 0 (default): from the lowest
                           diagonal determinant.  A parent state can overlap
                           an excited state of the child more than its
                           ground state, so the iteration can settle on the
                           wrong root; measured on the 8e/23o workload it
                           saved few iterations.                             */
  /* Mixed-precision Davidson (MBE_MIXED_BF16X3) convergence schedule:       */
  double mixed_stage_tol;  /* the tensor-core stage stops at this residual
                              times max(1, |theta|) (default 1e-5)           */
  double mixed_round_drop; /* each refinement round asks for its starting
                              exact residual times this (0 < x < 1, default
                              1e-2; the round stops earlier at the target)   */
  double mixed_rel_tol;    /* final target max(conv_tol_r, this times
                              max(1, |theta|)) on the exact residual (default
                              2e-7: above the floor that FP32 storage of the
                              CI vector sets, a few 1e-8 |H|)                */
  int pspace;              /* mixed mode: size of the P-space preconditioner,
                              the number of alpha-beta symmetric basis
                              functions of lowest diagonal energy whose block
                              of H + lambda S^2 is solved exactly in the
                              Davidson correction (0 = diagonal only; at most
                              128; capped at half the symmetric space;
                              default 128)                                   */
  int64_t wait_limit;      /* polls of an mbarrier a tensor-core kernel makes
                              before it gives up, sets its error word and
                              returns (the call then fails with MBE_ETIMEOUT);
                              a poll lasts at most about a microsecond;
                              default 2^24 (seconds); 0 gives up at the first
                              wait (for tests of the error path)             */
  int autotune;            /* 1: the first sigma call of each bin shape
                              (n, n_sigma) of the mixed mode times every
                              operand plan of the two-spin tensor-core kernel
                              that fits (A-operand stages 2..4, pull lists in
                              shared or global memory, one or two epilogue
                              groups) on its own data and
                              keeps the fastest for the shape; 0 (default):
                              the most stages that fit, lists in shared
                              memory when they fit.  All plans give the same
                              bits.                                          */
  const char* tune_file;   /* autotune cache (may be NULL): read at
                              mbe_create, one line per tuned shape appended
                              as it is tuned ("sigma_ab n nsig nstages
                              pull_smem groups ms"); the string is copied    */
  int graphs;              /* mixed mode: 1 (default) issues each Davidson
                              iteration (sigma vector, subspace update, Ritz
                              step, residual, correction and its
                              orthogonalisation) as one CUDA graph, captured
                              from the stream and replayed through an
                              executable graph updated in place; 0: plain
                              stream launches.  Same kernels, same bits.    */
} mbe_options;

typedef struct mbe_ctx mbe_ctx;

/* Counters accumulated by a context since creation or mbe_reset_stats. */
typedef struct mbe_stats {
  int64_t casci;          /* CASCI problems solved                            */
  int64_t sigma_vectors;  /* sigma-vector applications inside Davidson        */
  double sigma_flops;     /* algorithmic flops of the (kl|ij) contraction,
                             2 * N_det * npair^2 per sigma vector             */
  int64_t iters_total;    /* Davidson iterations summed over CASCIs           */
  int64_t iters_max;      /* largest iteration count of one CASCI             */
  int64_t noconv;         /* CASCIs that hit the iteration cap                */
  int64_t launches;       /* kernels the library ran on the device (those of
                             replayed CUDA graphs included)                   */
  int64_t dom_launches;   /* launches of the fused tensor-core sigma kernel   */
  double dom_ms;          /* their summed device time (CUDA events on the
                             context stream); 0 unless opt.timing = 1         */
  double dom_flops;       /* their algorithmic flops, 2 N_det npair^2 per
                             sigma vector                                     */
  int64_t fp64_launches;  /* launches of the FP64 (kl|ij) contraction kernel  */
  double fp64_ms;         /* their summed device time (opt.timing = 1)        */
  double fp64_flops;      /* their algorithmic flops                          */
  int64_t host_launches;  /* launch calls the host made: kernel launches
                             outside graphs plus graph launches               */
  int64_t graph_launches; /* CUDA graph launches (opt.graphs)                 */
  int64_t graph_builds;   /* graphs instantiated (the others were updated in
                             place before their launch)                       */
} mbe_stats;

/* Fill *opt with the defaults (FP64, max_batch 256, subspace 20, 400
 * iterations, tol_r 1e-8, tol_e 1e-12, spin_shift 0.5, keep_ci 0,
 * deterministic 1, no memory cap, warm_start 0, mixed schedule 1e-5 / 1e-2 /
 * 2e-7, pspace 128, wait_limit 2^24, autotune 0, graphs 1). */
void mbe_default_options(mbe_options* opt);

/* Create a context on CUDA device `device`.  opt may be NULL (defaults).
 * The context owns its device memory and a CUDA stream. */
int mbe_create(mbe_ctx** out, int device, const mbe_options* opt);
void mbe_destroy(mbe_ctx* ctx);

/* Make the context issue its work on `stream` (a cudaStream_t of the
 * context's device, caller-owned, must outlive its use); NULL restores the
 * context's own stream.  Lets a caller bracket the library's work with CUDA
 * events on a stream it knows. */
int mbe_set_stream(mbe_ctx* ctx, void* stream);
const char* mbe_last_error(const mbe_ctx* ctx);

/* Load the molecular integrals (input of every CASCI of Sec. 2).
 *  norb   number of spatial orbitals (1..128)
 *  nelec  number of (correlated) electrons; the reference determinant is
 *         the closed shell (even nelec) or the high-spin doublet (odd),
 *         see mbe_set_spin
 *  h      norb*norb, eri npair*npair (see conventions); NaN/Inf -> EINVAL.
 * Resets the reference space, the increment hash and kept RDMs. */
int mbe_load_integrals(mbe_ctx* ctx, int norb, int nelec, const double* h,
                       const double* eri);

/* Spin of the reference determinant (Fig. 2: case (a) closed shell, case
 * (b) high-spin open shell).  two_sz = n_alpha - n_beta >= 0 with the
 * parity of nelec: orbitals 0 .. n_beta - 1 are doubly occupied, n_beta ..
 * n_alpha - 1 singly occupied (alpha).  Every CASCI is then solved in the
 * determinant space of that Ms = two_sz / 2 for its lowest S = Ms state;
 * the singly occupied orbitals must belong to the reference space (checked
 * by mbe_set_reference, MBE_EINVAL), so the inactive core stays closed-shell.
 * Open-shell spaces run on the FP64 path (FP64-grade emulated contraction
 * in the mixed and emulated modes; the split-BF16x3 sigma and the
 * warm starts need alpha<->beta symmetric vectors).  MBE_EINVAL for a bad
 * two_sz, MBE_ESTATE before mbe_load_integrals.  Resets the reference. */
int mbe_set_spin(mbe_ctx* ctx, int two_sz);

/* Set the reference space Pi (Sec. 2, Eq. 3) and the expansion space.
 *  ref_orbs[nref]  orbitals of Pi (distinct, any order)
 *  exp_orbs[nexp]  expansion orbitals (distinct, disjoint from Pi)
 * Solves the order-0 CASCI of Pi; its energy is written to *e_ref (may be
 * NULL).  Resets the increment hash.  With a high-spin reference
 * (mbe_set_spin) Pi must hold every singly occupied orbital. */
int mbe_set_reference(mbe_ctx* ctx, const int* ref_orbs, int nref,
                      const int* exp_orbs, int nexp, double* e_ref);

/* Solve the CASCI of every tuple (Sec. 2: active space = Pi + tuple).
 *  order        tuple length n >= 1
 *  tuples       ntup*order expansion orbitals, each row strictly ascending
 *  e_out        ntup total CASCI energies eps_T (may be NULL)
 *  status_out   ntup per-tuple status (0 converged, MBE_ENOCONV) (may be NULL)
 * The tuples become the "current order" consumed by mbe_increments.
 * Returns MBE_ENOCONV if any tuple did not converge (energies still
 * written). */
int mbe_solve_tuples(mbe_ctx* ctx, int order, const int32_t* tuples,
                     int64_t ntup, double* e_out, int32_t* status_out);

/* Increments of the current order (Eq. 3) by hash lookup of all proper
 * non-empty subtuples (all lower orders must have been processed, in
 * order), insertion of the new increments, screening and the order sum.
 *  screen_thr  |increment| >= screen_thr marks a tuple "kept" (may spawn
 *              children); 0 keeps all
 *  inc_out     ntup increments (may be NULL)
 *  keep_out    ntup flags (may be NULL)
 *  e_order_out Kahan sum of the order's increments (may be NULL)
 *  e_total_out eps_Pi + Kahan sum of all order sums so far (may be NULL)
 * Returns MBE_ELOOKUP if a subtuple is missing. */
int mbe_increments(mbe_ctx* ctx, int order, double screen_thr, double* inc_out,
                   uint8_t* keep_out, double* e_order_out, double* e_total_out);

/* Tuples of order `order` (>= 2) generated on the device from the last
 * processed order by the screening rule: a tuple is formed iff every one of
 * its (order-1)-subtuples exists and at least one of them is kept.  For
 * order 1 every expansion orbital.  Lexicographic order.
 *  tuples_out  capacity cap rows of `order` int32 (may be NULL to count)
 *  ntup_out    number of tuples (always written)
 * Returns MBE_EINVAL if cap is too small (ntup_out still written). */
int mbe_next_tuples(mbe_ctx* ctx, int order, int32_t* tuples_out, int64_t cap,
                    int64_t* ntup_out);

/* pi-pruning (Sec. 3): restrict the expansion to tuples that hold both
 * orbitals of a given degenerate pair or neither.  The expansion then runs
 * over units (single orbitals and pairs): mbe_next_tuples forms a tuple of
 * order k (its orbital count) from a tuple with one unit fewer (order k-1 or
 * k-2; the empty tuple for a lone unit) by the screening rule applied to its
 * one-unit-removed subtuples, mbe_increments subtracts the increments of its
 * proper non-empty sub-unions of units (Eq. 3 over units) and the MBE
 * coefficients of mbe_energy_backward count units.  An order can be empty
 * while the next one is not (a pair adds two orbitals).
 *  pairs[2*npairs]  pairs of expansion orbitals (host); each orbital in at
 *                   most one pair; npairs = 0 switches pruning off
 * Call after mbe_set_reference and before the first order (MBE_ESTATE
 * otherwise); mbe_set_reference switches pruning off. */
int mbe_set_pruning_pairs(mbe_ctx* ctx, const int32_t* pairs, int npairs);

/* Gradient of the MBE energy (eps_Pi + all increments processed so far)
 * with respect to the integrals, by Hellmann-Feynman: each CASCI energy is
 * stationary in its CI coefficients, so dE/dh_pq = sum_T c_T gamma^T_pq and
 * dE/d(pq|rs) = 1/2 sum_T c_T Gamma^T_pqrs, with full-space spin-summed RDMs
 * (inactive core included) and c_T = sum_{U in set, U >= T} (-1)^{|U|-|T|}.
 * Needs keep_ci = 1 when the reference and the tuples were solved.  With
 * opt.backward_share = 0 a tuple with a non-zero c_T whose RDMs are not
 * held returns MBE_ESTATE; with 1 or 2 such tuples are skipped (they were
 * solved by another context) so that the outputs of all contexts sum to the
 * gradient.
 *  scale  multiplies the outputs (the incoming dL/dE)
 *  dh     norb*norb (symmetric)
 *  deri   npair*npair, gradient w.r.t. the symmetric packed eri matrix
 *         (sum over the full-tensor images of (P,Q), symmetrised P<->Q). */
int mbe_energy_backward(mbe_ctx* ctx, double scale, double* dh, double* deri);

/* Make `tuples` (ntup rows of `order` orbitals, ascending) with the given
 * CASCI energies eps (total, Eh) the current order, as mbe_solve_tuples
 * would, without solving.  Used when the tuples of one order are solved on
 * several GPUs: each process solves its share, the energies are gathered
 * and every process continues with mbe_increments on the full order.
 * Kept RDMs (keep_ci) of tuples this context solved for this order are
 * retained. */
int mbe_set_order_energies(mbe_ctx* ctx, int order, const int32_t* tuples,
                           int64_t ntup, const double* eps);

/* Copy the context's counters to *out (host). */
int mbe_get_stats(const mbe_ctx* ctx, mbe_stats* out);
/* Zero the context's counters. */
int mbe_reset_stats(mbe_ctx* ctx);

/* Sigma vector of one CASCI for testing: sigma = (H_active + spin_shift*S^2)
 * c in the determinant basis of strings (Ia, Ib), in the context precision.
 *  act[nact]  active orbitals; c, sigma  nstr_alpha*nstr_beta (host),
 *             index Ia*nstr_beta + Ib (nstr_alpha = nstr_beta for a closed
 *             shell; a high-spin reference, mbe_set_spin, needs its singly
 *             occupied orbitals in act)
 * H_active excludes the inactive-core energy (returned in *e_core). */
int mbe_sigma(mbe_ctx* ctx, const int* act, int nact, const double* c,
              double* sigma, double* e_core);

/* Device scratch of mbe_sigma_noalloc, per device (16 MiB). */
#define MBE_NOALLOC_SCRATCH_BYTES (16u << 20)

/* mbe_sigma without device-memory allocation (the paper has no counterpart;
 * it serves callers that may not allocate: cudaMalloc / cudaFree can
 * synchronise the whole device, and a caller under a fixed device-memory
 * budget cannot let the context's pool grow).  Always the FP64 sigma
 * (H_active + spin_shift*S^2) c, whatever opt.precision says; closed-shell
 * references only (MBE_EINVAL after mbe_set_spin with two_sz > 0).
 *  act[nact]   active orbitals (host)
 *  c_dev       nstr*nstr doubles, DEVICE memory of the context's device,
 *              caller-owned, read only
 *  sigma_dev   nstr*nstr doubles, DEVICE memory, caller-owned, fully
 *              overwritten (need not be zeroed)
 *  ndet        element count of c_dev and sigma_dev; MBE_EINVAL unless it
 *              equals nstr*nstr of the active space
 *  e_core      host; if non-NULL the inactive-core energy is written there
 *              and the call waits for the context stream; if NULL the call
 *              returns once the work is enqueued on the context stream.
 * All intermediates (string tables, effective integrals, the D and E
 * intermediates of the sigma) live in one file-scope device array of
 * MBE_NOALLOC_SCRATCH_BYTES per device; none of it needs to start at zero.
 * A problem that does not fit (roughly more than 9 active orbitals) returns
 * MBE_EINVAL and launches nothing.  Calls overlapping on one device race on
 * that array: issue them on one stream or wait for one before the next.
 * The first call on a device looks the array up (cudaGetSymbolAddress),
 * sets a kernel attribute and copies a small constant table with a
 * synchronous cudaMemcpyToSymbol (once per device, shared with the other
 * entry points); make it before any stream capture.  The active orbitals
 * reach the device as a kernel argument; with e_core non-NULL the call
 * copies the core energy to the host and waits for the stream. */
int mbe_sigma_noalloc(mbe_ctx* ctx, const int* act, int nact, const double* c_dev,
                      double* sigma_dev, int64_t ndet, double* e_core);

/* Arithmetic peaks of CUDA device `device` measured by the library (no
 * counterpart in the paper; a measurement aid for rooflines): FMA throughput
 * of CUDA-core FP64 and FP32 arithmetic in TFLOP/s (2 flops per FMA), from
 * probe kernels of independent FMA chains on 8 CTAs per SM timed with CUDA
 * events (best of three launches after a warm-up).  Takes well under a
 * second; allocates a small output buffer with cudaMalloc.
 *  fp64_tflops, fp32_tflops  host outputs (either may be NULL) */
int mbe_measure_peaks(int device, double* fp64_tflops, double* fp32_tflops);

#ifdef __cplusplus
}
#endif
#endif /* MBE_H */
