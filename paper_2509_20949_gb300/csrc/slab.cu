// slab.cu -- lattice decomposition along z (Sec. 2.2, lattice parallelism):
// the per-sweep plan of each rank, the planes that move between ranks when the
// link-cell grid moves, and the merge kernel of the boundary planes.
#include <cstdint>
#include <string>

#include "kernels.h"
#include "smcx.h"
#include "smcx_common.cuh"

namespace smcx {
smcx_status batch_fail(smcx_status s, const std::string& msg);
void host_layout(const smcx_lattice_desc& d, int M, int* L, int m[3]);
bool host_desc_ok(const smcx_lattice_desc* d, std::string* why);
void host_sweep_origin(const smcx_lattice_desc& d, uint32_t t, int shift[3]);

// occupancy ^= theirs ^ before, 16 bytes per thread
__global__ void k_merge_planes(uint4* __restrict__ occ, const uint4* __restrict__ theirs,
                               const uint4* __restrict__ before, size_t n16) {
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n16;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const uint4 a = occ[i], b = theirs[i], c = before[i];
    occ[i] = make_uint4(a.x ^ b.x ^ c.x, a.y ^ b.y ^ c.y, a.z ^ b.z ^ c.z, a.w ^ b.w ^ c.w);
  }
}

cudaError_t launch_merge_planes(uint8_t* occ, const uint8_t* theirs, const uint8_t* before,
                                size_t bytes, int n_sm, cudaStream_t st) {
  const size_t n16 = bytes / 16;
  if (n16 == 0) return cudaSuccess;
  size_t blocks = (n16 + 255) / 256;
  const size_t cap = static_cast<size_t>(n_sm > 0 ? n_sm : 152) * 8;
  if (blocks > cap) blocks = cap;
  k_merge_planes<<<static_cast<unsigned>(blocks), 256, 0, st>>>(
      reinterpret_cast<uint4*>(occ), reinterpret_cast<const uint4*>(theirs),
      reinterpret_cast<const uint4*>(before), n16);
  return cudaGetLastError();
}
}  // namespace smcx

namespace {

using smcx::batch_fail;

struct Plan {
  int c_lo, c_hi, z_lo, n_own, halo, m_z, n_z;
};

smcx_status plan_of(const smcx_lattice_desc* desc, uint32_t n_shells, uint32_t world,
                    uint32_t rank, uint32_t t, Plan* p) {
  std::string why;
  if (!desc || !smcx::host_desc_ok(desc, &why))
    return batch_fail(SMCX_EINVAL, desc ? why : std::string("null descriptor"));
  if (n_shells < 1 || n_shells > static_cast<uint32_t>(smcx::kMaxShells))
    return batch_fail(SMCX_EINVAL, "n_shells must be 1..4");
  if (world == 0 || rank >= world) return batch_fail(SMCX_EINVAL, "need rank < world");
  int L = 0, m[3];
  smcx::host_layout(*desc, static_cast<int>(n_shells), &L, m);
  const int mz = m[2];
  if (world > 1 && mz < 2 * static_cast<int>(world))
    return batch_fail(SMCX_EINVAL, "each rank needs two link-cell planes or more (m_z >= 2 world)");
  const int nz = static_cast<int>(desc->n[2]);
  int shift[3];
  smcx::host_sweep_origin(*desc, t, shift);
  auto bound = [&](int c) { return static_cast<int>((static_cast<int64_t>(c) * nz) / mz); };
  p->c_lo = static_cast<int>((static_cast<int64_t>(rank) * mz) / world);
  p->c_hi = static_cast<int>((static_cast<int64_t>(rank + 1) * mz) / world);
  p->z_lo = (shift[2] + bound(p->c_lo)) % nz;
  p->n_own = bound(p->c_hi) - bound(p->c_lo);
  p->halo = L;
  p->m_z = mz;
  p->n_z = nz;
  return SMCX_OK;
}

}  // namespace

extern "C" {

smcx_status smcx_slab_plan(const smcx_lattice_desc* desc, uint32_t n_shells, uint32_t world,
                           uint32_t rank, uint32_t t, smcx_slab* out) {
  if (!out) return batch_fail(SMCX_EINVAL, "null output");
  Plan p;
  const smcx_status s = plan_of(desc, n_shells, world, rank, t, &p);
  if (s != SMCX_OK) return s;
  out->c_lo = p.c_lo;
  out->c_hi = p.c_hi;
  out->z_lo = p.z_lo;
  out->n_own = p.n_own;
  out->halo = p.halo;
  out->m_z = p.m_z;
  return SMCX_OK;
}

// owned(from, t) intersected with window(to, t + 1) on the circle of n_z
// planes: both arcs are at most n_z long (a window is n_own + 2 halo <= n_z
// when world > 1, since the other ranks own 2 halo planes or more), so the
// intersection is at most two runs.
smcx_status smcx_slab_transfer(const smcx_lattice_desc* desc, uint32_t n_shells, uint32_t world,
                               uint32_t from, uint32_t to, uint32_t t, int32_t* runs,
                               uint32_t* n_runs) {
  if (!runs || !n_runs) return batch_fail(SMCX_EINVAL, "null output");
  if (to >= world) return batch_fail(SMCX_EINVAL, "need to < world");
  Plan a, b;
  smcx_status s = plan_of(desc, n_shells, world, from, t, &a);
  if (s != SMCX_OK) return s;
  s = plan_of(desc, n_shells, world, to, t + 1, &b);
  if (s != SMCX_OK) return s;
  *n_runs = 0;
  if (from == to) return SMCX_OK;
  const int n = a.n_z;
  const int a0 = a.z_lo, a1 = a.z_lo + a.n_own;               // [a0, a1), a0 in [0, n)
  const int w0 = ((b.z_lo - b.halo) % n + n) % n;               // window start in [0, n)
  const int wl = b.n_own + 2 * b.halo;
  if (wl > n || a.n_own > n) return batch_fail(SMCX_EINVAL, "internal: arc longer than n_z");
  int found[3][2], nf = 0;
  for (int k = -1; k <= 1; ++k) {
    const int b0 = w0 + k * n, b1 = b0 + wl;
    const int lo = a0 > b0 ? a0 : b0, hi = a1 < b1 ? a1 : b1;
    if (hi > lo) {
      found[nf][0] = lo;
      found[nf][1] = hi - lo;
      ++nf;
    }
  }
  // join runs that meet (adjacent on the unrolled line), then reduce mod n
  int outn = 0;
  for (int i = 0; i < nf; ++i) {
    if (outn > 0 && runs[2 * (outn - 1)] + runs[2 * (outn - 1) + 1] == found[i][0]) {
      runs[2 * (outn - 1) + 1] += found[i][1];
      continue;
    }
    if (outn == 2) return batch_fail(SMCX_EINVAL, "internal: more than two runs");
    runs[2 * outn] = found[i][0];
    runs[2 * outn + 1] = found[i][1];
    ++outn;
  }
  for (int i = 0; i < outn; ++i) runs[2 * i] = ((runs[2 * i] % n) + n) % n;
  *n_runs = static_cast<uint32_t>(outn);
  return SMCX_OK;
}

}  // extern "C"
