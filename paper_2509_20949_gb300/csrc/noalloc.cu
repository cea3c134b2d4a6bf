// noalloc.cu -- directed shell pair counts without any allocation.
//
// Some callers cannot allocate device memory at the point where they need
// the Warren-Cowley pair counts: code that runs inside another framework's
// memory-pool callbacks or allocator hooks (where a nested allocation would
// recurse or deadlock), processes whose device memory is entirely reserved
// by their host framework, and embedded or real-time users that forbid
// allocation after start-up.  For them smcx_pair_counts_noalloc takes the
// occupancy and the output as device pointers and keeps its accumulators in
// a static device array of this file (SMCX_NOALLOC_MAX_SHELLS x
// SMCX_NOALLOC_MAX_SPECIES^2 counters, 8 KiB), which every GPU that loads
// the library holds until the process exits.  It is a variant of the
// generic pair-count kernel: same counting, canonical site indexing, the
// static array as its scratch.
#include <string>

#include "../../include/smcx.h"
#include "smcx_common.cuh"

namespace smcx {
smcx_status batch_fail(smcx_status s, const std::string& msg);  // sets smcx_last_error()
}

namespace {

using namespace smcx;

constexpr int kMaxShellsNA = SMCX_NOALLOC_MAX_SHELLS;
constexpr int kMaxSpeciesNA = SMCX_NOALLOC_MAX_SPECIES;
constexpr int kScratchCounters = kMaxShellsNA * kMaxSpeciesNA * kMaxSpeciesNA;

// the scratch: shared by every call on a device (see smcx.h)
static __device__ __align__(256) unsigned long long g_na_scratch[kScratchCounters];

struct NaGeom {
  int kind, nb;
  int n[3];
  int K;
  int n_shells;
  int8_t v[kMaxShellVecs][3];
  int start[kMaxShells + 1];
};

__device__ __forceinline__ int na_mod(int a, int n) {
  const int r = a % n;
  return r < 0 ? r + n : r;
}

__global__ void k_na_clear(unsigned long long* __restrict__ scratch, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    scratch[i] = 0ull;
}

// N_m[p'][p] over every site of the canonical occupancy (site index
// ((z*ny + y)*nx + x)*nb + b), block counters in shared memory
__global__ void __launch_bounds__(256) k_na_pair_count(const NaGeom g,
                                                       const uint8_t* __restrict__ canon,
                                                       unsigned long long* __restrict__ scratch,
                                                       uint32_t n_sites) {
  __shared__ uint32_t s_cnt[kScratchCounters];
  const int K = g.K;
  const int n_cnt = g.n_shells * K * K;
  for (int c = threadIdx.x; c < n_cnt; c += blockDim.x) s_cnt[c] = 0;
  __syncthreads();
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_sites;
       i += gridDim.x * blockDim.x) {
    const int b = static_cast<int>(i % g.nb);
    const uint32_t cell = i / g.nb;
    const int x = static_cast<int>(cell % g.n[0]);
    const int y = static_cast<int>((cell / g.n[0]) % g.n[1]);
    const int z = static_cast<int>(cell / (static_cast<uint32_t>(g.n[0]) * g.n[1]));
    const uint32_t pc = canon[i];
    if (pc >= static_cast<uint32_t>(K)) continue;  // ids >= K are not counted
    for (int m = 0; m < g.n_shells; ++m)
      for (int t = g.start[m]; t < g.start[m + 1]; ++t) {
        const int hx = na_mod(2 * x + basis_comp(g.kind, b, 0) + g.v[t][0], 2 * g.n[0]);
        const int hy = na_mod(2 * y + basis_comp(g.kind, b, 1) + g.v[t][1], 2 * g.n[1]);
        const int hz = na_mod(2 * z + basis_comp(g.kind, b, 2) + g.v[t][2], 2 * g.n[2]);
        const int bp = basis_of_parity(g.kind, hx & 1, hy & 1, hz & 1);
        const uint32_t k =
            ((static_cast<uint32_t>(hz >> 1) * g.n[1] + (hy >> 1)) * g.n[0] + (hx >> 1)) * g.nb + bp;
        const uint32_t q = canon[k];
        if (q < static_cast<uint32_t>(K)) atomicAdd(&s_cnt[(m * K + pc) * K + q], 1u);
      }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < n_cnt; c += blockDim.x)
    if (s_cnt[c]) atomicAdd(&scratch[c], static_cast<unsigned long long>(s_cnt[c]));
}

__global__ void k_na_copy(const unsigned long long* __restrict__ scratch,
                          unsigned long long* __restrict__ out, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = scratch[i];
}

// Device address of the scratch in the current device's current context.
// In host code g_na_scratch names a host-side stand-in, not device memory, so
// the address is asked of the runtime -- on every call, with the caller's
// device current: a symbol's address belongs to one context, and an address
// kept from an earlier call could point into a context that cudaDeviceReset
// (or a switch of context) has since destroyed.  The query is a host-side
// lookup; the first one on a device loads the library's module there.
smcx_status na_scratch_address(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
  if (e != cudaSuccess || !p)
    return smcx::batch_fail(SMCX_ECUDA,
                            std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  *out = p;
  return SMCX_OK;
}

}  // namespace

extern "C" smcx_status smcx_pair_counts_noalloc(uint32_t kind, const uint32_t* n,
                                                uint32_t n_species, uint32_t n_shells,
                                                const uint8_t* d_canon, uint64_t* d_counts,
                                                void* cuda_stream) {
  using smcx::batch_fail;
  if (kind > 1 || !n || !d_canon || !d_counts)
    return batch_fail(SMCX_EINVAL, "pair_counts_noalloc: bad kind or null pointer");
  if (n_species < 1 || n_species > SMCX_NOALLOC_MAX_SPECIES)
    return batch_fail(SMCX_EINVAL, "pair_counts_noalloc: n_species must be 1..16 (static scratch)");
  if (n_shells < 1 || n_shells > SMCX_NOALLOC_MAX_SHELLS)
    return batch_fail(SMCX_EINVAL, "pair_counts_noalloc: n_shells must be 1..4 (static scratch)");
  for (int d = 0; d < 3; ++d)
    if (n[d] < 1 || n[d] > (1u << 20)) return batch_fail(SMCX_EINVAL, "pair_counts_noalloc: bad n");
  const uint64_t sites = static_cast<uint64_t>(kind == 0 ? 2 : 4) * n[0] * n[1] * n[2];
  if (sites >= (1ull << 32)) return batch_fail(SMCX_EINVAL, "pair_counts_noalloc: too many sites");
  void* scratch = nullptr;
  smcx_status s = na_scratch_address(&scratch);
  if (s != SMCX_OK) return s;
  NaGeom g;
  g.kind = static_cast<int>(kind);
  g.nb = basis_count(g.kind);
  for (int d = 0; d < 3; ++d) g.n[d] = static_cast<int>(n[d]);
  g.K = static_cast<int>(n_species);
  g.n_shells = static_cast<int>(n_shells);
  for (int i = 0; i < shell_start(g.kind, kMaxShells); ++i) {
    const ShellVec v = shell_vec(g.kind, i);
    g.v[i][0] = v.x;
    g.v[i][1] = v.y;
    g.v[i][2] = v.z;
  }
  for (int m = 0; m <= kMaxShells; ++m) g.start[m] = shell_start(g.kind, m);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  auto* acc = static_cast<unsigned long long*>(scratch);
  const int n_cnt = static_cast<int>(n_shells * n_species * n_species);
  int dev = 0, n_sm = 148;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  uint64_t blocks = (sites + 255) / 256;
  if (blocks > static_cast<uint64_t>(n_sm) * 8) blocks = static_cast<uint64_t>(n_sm) * 8;
  k_na_clear<<<1, 256, 0, st>>>(acc, n_cnt);
  k_na_pair_count<<<static_cast<unsigned>(blocks), 256, 0, st>>>(g, d_canon, acc,
                                                                 static_cast<uint32_t>(sites));
  k_na_copy<<<1, 256, 0, st>>>(acc, reinterpret_cast<unsigned long long*>(d_counts), n_cnt);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return batch_fail(SMCX_ECUDA, std::string("pair_counts_noalloc: ") + cudaGetErrorString(e));
  return SMCX_OK;
}
