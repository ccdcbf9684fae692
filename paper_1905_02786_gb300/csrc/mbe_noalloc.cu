// mbe_sigma_noalloc: the FP64 sigma vector of mbe_sigma with every
// intermediate in one file-scope device array instead of the context's pool.
//
// Callers it serves: code that must not allocate device memory around a
// sigma application -- cudaMalloc and cudaFree can synchronise the whole
// device (stalling every other stream of the process), and a caller running
// under a fixed device-memory budget (the rest of HBM held by another
// allocator) cannot let the pool grow.  This path calls no allocating
// routine; it reads integrals, writes into the caller's device buffers and
// the scratch array below.
//
// Scratch: MBE_NOALLOC_SCRATCH_BYTES per device (the array is part of the
// loaded module, one copy per device).  A problem whose tables, integrals
// and D / E intermediates do not fit is rejected with MBE_EINVAL before
// anything is launched.  No part of the scratch needs to start at zero:
// every word a kernel reads is written earlier in the same call (string
// tables, effective integrals, D by the gather, E by the contraction).
//
// Calls that overlap on one device race on the single scratch array: a
// caller serialises them (issue them on one stream, or wait for one call to
// finish before issuing the next from another stream or context).
//
// The first call on a device resolves the scratch address with
// cudaGetSymbolAddress and sets the contraction kernel's shared-memory
// attribute; it should come before any stream capture.  The active orbitals
// reach the scratch through a kernel argument (no host-memory copy); with a
// non-NULL e_core the call copies the core energy back and waits for the
// stream.
#include "mbe_internal.cuh"
#include <algorithm>
#include <mutex>

namespace {

static __device__ __align__(256) unsigned char g_sigma_scratch[MBE_NOALLOC_SCRATCH_BYTES];

std::mutex g_scratch_mu;
void* g_scratch_ptr[MBE_MAX_DEVICES] = {nullptr};

unsigned char* scratch_base(int device) {
  if (device < 0 || device >= MBE_MAX_DEVICES) throw MbeError{MBE_EINVAL, "device index out of range"};
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    CU_CHECK(cudaGetSymbolAddress(&p, g_sigma_scratch));
    if (!p) throw MbeError{MBE_ECUDA, "scratch symbol has no device address"};
    g_scratch_ptr[device] = p;
  }
  return (unsigned char*)g_scratch_ptr[device];
}

// byte offsets of the pieces inside the scratch array (256-byte aligned)
struct NoallocLayout {
  size_t masks, link, act, bmap, ecore, heff, hp, gp, jk, D, E, total;
};

NoallocLayout noalloc_layout(int n, int64_t nstr) {
  const int64_t npair = (int64_t)n * (n + 1) / 2;
  const int64_t ndet = nstr * nstr;
  NoallocLayout L;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t r = o;
    o += (bytes + 255) & ~(size_t)255;
    return r;
  };
  L.masks = take(sizeof(uint32_t) * nstr);
  L.link = take(sizeof(int32_t) * nstr * npair);
  L.act = take(sizeof(int32_t) * n);
  L.bmap = take(sizeof(int32_t));
  L.ecore = take(sizeof(double));
  L.heff = take(sizeof(double) * n * n);
  L.hp = take(sizeof(double) * n * n);
  L.gp = take(sizeof(double) * npair * npair);
  L.jk = take(sizeof(double) * 2 * n * n);
  L.D = take(sizeof(double) * npair * ndet);
  L.E = take(sizeof(double) * npair * ndet);
  L.total = o;
  return L;
}

// the sorted active orbitals (at most 15) passed by value
struct ActList {
  int32_t v[16];
};
__global__ void k_put_act(ActList a, int n, int32_t* __restrict__ dst, int32_t* __restrict__ bmap) {
  const int t = threadIdx.x;
  if (t < n) dst[t] = a.v[t];
  if (t == 0) bmap[0] = 0;
}

}  // namespace

int noalloc_sigma_run(mbe_ctx* ctx, const int* act, int nact, const double* c_dev,
                      double* sigma_dev, int64_t ndet_arg, double* e_core) {
  if (ctx->norb == 0) throw MbeError{MBE_ESTATE, "no integrals loaded"};
  if (nact < 1 || nact > 15 || !act || !c_dev || !sigma_dev)
    throw MbeError{MBE_EINVAL, "bad sigma arguments"};
  if (ctx->two_sz != 0)
    throw MbeError{MBE_EINVAL, "the no-allocation sigma takes closed-shell references only"};
  std::vector<int32_t> a(act, act + nact);
  std::sort(a.begin(), a.end());
  for (int i = 0; i < nact; i++)
    if (a[i] < 0 || a[i] >= ctx->norb || (i && a[i] == a[i - 1]))
      throw MbeError{MBE_EINVAL, "bad active orbital"};
  int nsig = 0;
  for (int o : a) nsig += o < ctx->nocc;
  const int64_t nstr = string_count(nact, nsig);
  if (ndet_arg != nstr * nstr)
    throw MbeError{MBE_EINVAL, "vector length does not match the active space"};
  const NoallocLayout L = noalloc_layout(nact, nstr);
  if (L.total > (size_t)MBE_NOALLOC_SCRATCH_BYTES)
    throw MbeError{MBE_EINVAL, "active space too large for the no-allocation scratch"};
  unsigned char* base = scratch_base(ctx->device);
  uint32_t* masks = (uint32_t*)(base + L.masks);
  int32_t* link = (int32_t*)(base + L.link);
  int32_t* actd = (int32_t*)(base + L.act);
  int32_t* bmap = (int32_t*)(base + L.bmap);
  double* ecore = (double*)(base + L.ecore);
  cudaStream_t st = ctx->stream;
  ActList al = {};
  for (int i = 0; i < nact; i++) al.v[i] = a[i];
  k_put_act<<<1, 32, 0, st>>>(al, nact, actd, bmap);
  CU_LAUNCH_CHECK();
  launch_string_tables(ctx, nact, nsig, (int)nstr, masks, link);
  launch_effints_raw(ctx, actd, 1, nact, 2 * nsig, ecore, (double*)(base + L.heff),
                     (double*)(base + L.hp), (double*)(base + L.gp), (double*)(base + L.jk));
  const int64_t ndet = nstr * nstr;
  sigma_fp64_raw(ctx, nact, nsig, (int)nstr, link, masks, (const double*)(base + L.gp), c_dev, ndet,
                 sigma_dev, ndet, nullptr, bmap, 1, (double*)(base + L.D), (double*)(base + L.E),
                 ctx->opt.spin_shift, false, nullptr);
  if (e_core) {
    CU_CHECK(cudaMemcpyAsync(e_core, ecore, sizeof(double), cudaMemcpyDeviceToHost, st));
    CU_CHECK(cudaStreamSynchronize(st));
  }
  return MBE_OK;
}
