// smcx_capi.cu -- the C ABI of libsmcx.so (include/smcx.h): validation, the
// link-cell layout, the per-sweep schedule (origin shift, colours, Metropolis
// threshold tables) and kernel launches.  Host code only; the kernels live in
// kernels_*.cu.
#include <array>
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/smcx.h"
#include "kernels.h"
#include "trace.h"

using namespace smcx;

namespace {

thread_local std::string g_err;

smcx_status fail(smcx_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

// Boltzmann constant in eV/K (CODATA 2018); the paper (Sec. 2.1) uses
// beta = 1/(k_B T) without a value.
constexpr double kBoltzmannEvPerK = 8.617333262e-5;

bool desc_ok(const smcx_lattice_desc* d, std::string* why) {
  if (!d) {
    *why = "null descriptor";
    return false;
  }
  if (d->kind != SMCX_BCC && d->kind != SMCX_FCC) {
    *why = "kind must be SMCX_BCC or SMCX_FCC";
    return false;
  }
  for (int c = 0; c < 3; ++c)
    if (d->n[c] < 1 || d->n[c] > (1u << 20)) {
      *why = "n[] must be in 1..2^20";
      return false;
    }
  if (d->pack_bits != 8 && d->pack_bits != 4) {
    *why = "pack_bits must be 8 or 4";
    return false;
  }
  const uint32_t kmax = d->pack_bits == 4 ? 16u : 255u;
  if (d->n_species < 1 || d->n_species > kmax) {
    *why = "n_species out of range (1..255, 1..16 when packed)";
    return false;
  }
  const uint64_t N = static_cast<uint64_t>(basis_count(static_cast<int>(d->kind))) * d->n[0] *
                     d->n[1] * d->n[2];
  if (N >= (1ull << 32)) {
    *why = "lattice has 2^32 or more sites";
    return false;
  }
  if (d->min_cell > (1u << 20)) {
    *why = "min_cell too large";
    return false;
  }
  if (d->flags & ~(SMCX_NO_SHIFT | SMCX_SINGLE_CELL)) {
    *why = "unknown flag bits";
    return false;
  }
  return true;
}

uint64_t n_sites(const smcx_lattice_desc* d) {
  return static_cast<uint64_t>(basis_count(static_cast<int>(d->kind))) * d->n[0] * d->n[1] *
         d->n[2];
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

size_t row_pitch(const smcx_lattice_desc* d) { return align_up(d->n[0], 16); }

// device storage: [group][z][y] rows of row_pitch bytes (see Geom in
// smcx_common.cuh); groups = basis sites (8-bit) or basis pairs (4-bit)
size_t occ_bytes(const smcx_lattice_desc* d) {
  const size_t nb = static_cast<size_t>(basis_count(static_cast<int>(d->kind)));
  const size_t groups = d->pack_bits == 4 ? nb / 2 : nb;
  return groups * d->n[2] * d->n[1] * row_pitch(d);
}

struct WorkLayout {
  size_t stats;    // 16 x u64: call stats, cumulative stats, status/flags
  size_t V;        // [4][K][K] int64
  size_t D;        // per-(p, q) difference rows of the tiled kernel
  size_t pairs;    // [4][K][K] u64
  size_t local;    // K <= 8: LocalParam, the local-energy table, energy partial sums
  size_t scratch;  // N bytes: canonical occupancy in transit
  size_t total;
};

constexpr int kLocalPartials = 2048;  // blocks of the local-energy reduction
constexpr size_t kLocalParamOff = 0;
constexpr size_t kLocalTableOff = (sizeof(LocalParam) + 255) / 256 * 256;

size_t local_table_bytes(size_t K) {
  return sizeof(int64_t) * kLocalMaxShells * K * K * kLocalMaxZT;
}

size_t local_bytes(size_t K) {
  if (K > static_cast<size_t>(kLocalMaxK)) return 0;
  return kLocalTableOff + align_up(local_table_bytes(K), 256) +
         align_up(sizeof(long long) * kLocalPartials, 256);
}

constexpr size_t kTiledTableWords = 6 * 6 * 160 / 4;  // largest table: K = 6, M = 4

WorkLayout work_layout(const smcx_lattice_desc* d) {
  const size_t K = d->n_species;
  WorkLayout w;
  w.stats = 0;
  w.V = 256;
  w.D = w.V + align_up(sizeof(int64_t) * kMaxShells * K * K, 256);
  w.pairs = w.D + align_up(sizeof(uint32_t) * kTiledTableWords, 256);
  const size_t kp = K < 6 ? 6 : K;  // the tiled pair count writes [4][6][6] at most
  w.local = w.pairs + align_up(sizeof(uint64_t) * kMaxShells * kp * kp, 256);
  w.scratch = w.local + local_bytes(K);
  w.total = w.scratch + align_up(static_cast<size_t>(n_sites(d)), 256);
  return w;
}

// Threshold tables of the Metropolis test (Sec. 2.1, Eq. 3) at temperature T:
// bins of width 2^s q (q = 2^-32 eV) with beta q 2^s <= 2^-20, evaluated at
// their lower edge, exp(-beta q 2^s idx) = T_0[idx & 511] T_1[(idx>>9)&511]
// T_2[idx>>18] in 2^32 fixed point.
bool build_tables(double T, Tables* tab, int* mode, int* s) {
  if (std::isnan(T) || T < 0) return false;
  std::memset(tab->w, 0, sizeof(tab->w));
  *s = 0;
  if (T == 0.0) {
    *mode = kModeZeroT;
    return true;
  }
  if (std::isinf(T)) {
    *mode = kModeAcceptAll;
    return true;
  }
  const double beta = 1.0 / (kBoltzmannEvPerK * T);
  if (beta == 0.0) {
    *mode = kModeAcceptAll;
    return true;
  }
  *mode = kModeNormal;
  const double limit = std::ldexp(1.0, -20);
  int sh = 0;
  while (sh < 62 && std::ldexp(beta, sh - 31) <= limit) ++sh;  // beta*2^((sh+1)-32)
  *s = sh;
  for (int level = 0; level < 3; ++level) {
    const double bin = std::ldexp(beta, sh - 32 + 9 * level);
    for (int i = 0; i < 512; ++i) {
      const double e = std::exp(-(static_cast<double>(i) * bin));
      double v = std::rint(std::ldexp(e, 32));
      if (v > 4294967295.0) v = 4294967295.0;
      tab->w[level * 512 + i] = static_cast<uint32_t>(v);
    }
  }
  return true;
}

// Per-sweep origin of the link-cell grid ("dynamically constructed" cells,
// Sec. 2.2): Philox counter (0, 0, t, 1); s_d = (w_d n_d) >> 32.
void sweep_origin(const smcx_lattice_desc& d, uint32_t t, int shift[3]) {
  if (d.flags & SMCX_NO_SHIFT) {
    shift[0] = shift[1] = shift[2] = 0;
    return;
  }
  const U4 w = philox4x32_10(0u, 0u, t, 1u, static_cast<uint32_t>(d.seed),
                             static_cast<uint32_t>(d.seed >> 32));
  const uint32_t ws[3] = {w.x, w.y, w.z};
  for (int c = 0; c < 3; ++c)
    shift[c] = static_cast<int>((static_cast<uint64_t>(ws[c]) * d.n[c]) >> 32);
}

int shell_reach(int kind, int M) {
  int r = 0;
  const int total = shell_start(kind, M);
  for (int i = 0; i < total; ++i) {
    const ShellVec v = shell_vec(kind, i);
    r = std::max(r, std::max(std::abs(v.x), std::max(std::abs(v.y), std::abs(v.z))));
  }
  return r;
}

}  // namespace

struct smcx_lattice {
  smcx_lattice_desc desc;
  int nb = 0;
  uint64_t N = 0;
  uint8_t* d_occ = nullptr;
  uint8_t* d_work = nullptr;
  cudaStream_t stream = nullptr;
  WorkLayout wl{};
  bool has_epi = false;
  uint32_t M = 0;
  std::vector<int64_t> V;
  int L = 0;
  int m[3] = {1, 1, 1};
  uint32_t t = 0;
  int64_t E0 = 0;         // energy when the running energy was last restarted
  bool e0_known = false;  // E0 was taken (at the last restart with a model, or a restore)
  smcx_status sticky = SMCX_OK;
  int opt_kernel = 0;
  int opt_tile = -1;
  int opt_staging = 0;
  int n_sm = 0;
  bool tiled_table_ok = false;  // the tiled kernel's int32 difference table fits
  bool local = false;           // the local-energy model replaces the EPI model
  int zt = 0;                   // its table's count axis
  int n_T = 0;                  // its table's entries
  int n_items = 0;              // its bystander (site, shell) items per direction
  bool t32 = false;             // every table entry fits int32
  int tiled_kmax = 0;
  // online kernel choice (SMCX_OPT_KERNEL = 0 and SMCX_OPT_TILE = -1): the
  // candidates (kernel, tile shape), the fastest phase seen for each, and
  // the phases timed so far
  struct Tuning {
    bool done = false;
    std::vector<std::pair<int, int>> cands;
    std::vector<float> best_ms;
    std::vector<int> samples;
    uint64_t next = 0;
    int choice = 0;
    std::vector<cudaEvent_t> ev;
  } tune;

  // asynchronous read-back (smcx_get_occupancy_async): copy stream, the
  // events after the conversion and after the copy, and whether a copy was
  // started and not yet waited for
  cudaStream_t copy = nullptr;
  cudaEvent_t ev_conv = nullptr, ev_down = nullptr;
  bool down_pending = false;

  ~smcx_lattice() {
    for (cudaEvent_t e : tune.ev) cudaEventDestroy(e);
    if (copy) cudaStreamSynchronize(copy);
    if (ev_conv) cudaEventDestroy(ev_conv);
    if (ev_down) cudaEventDestroy(ev_down);
    if (copy) cudaStreamDestroy(copy);
  }

  unsigned long long* stats() { return reinterpret_cast<unsigned long long*>(d_work + wl.stats); }
  int64_t* dV() { return reinterpret_cast<int64_t*>(d_work + wl.V); }
  unsigned long long* pairs() {
    return reinterpret_cast<unsigned long long*>(d_work + wl.pairs);
  }
  uint8_t* scratch() { return d_work + wl.scratch; }
  uint32_t* dtab() { return reinterpret_cast<uint32_t*>(d_work + wl.D); }
  unsigned int* flag() { return reinterpret_cast<unsigned int*>(stats() + kStatStatus); }
  LocalParam* dlp() { return reinterpret_cast<LocalParam*>(d_work + wl.local + kLocalParamOff); }
  int64_t* dT() { return reinterpret_cast<int64_t*>(d_work + wl.local + kLocalTableOff); }
  long long* dpart() {
    return reinterpret_cast<long long*>(d_work + wl.local + kLocalTableOff +
                                        align_up(local_table_bytes(desc.n_species), 256));
  }
  Geom geom() const;
};

namespace {

Geom geom_of(const smcx_lattice_desc& desc, int M, int L, const int m[3]) {
  Geom g;
  g.kind = static_cast<int>(desc.kind);
  g.nb = basis_count(g.kind);
  for (int c = 0; c < 3; ++c) {
    g.n[c] = static_cast<int>(desc.n[c]);
    g.m[c] = m[c];
  }
  g.L = L;
  g.K = static_cast<int>(desc.n_species);
  g.M = M;
  g.z1 = shell_z(g.kind, 0);
  g.pack4 = desc.pack_bits == 4;
  g.px = static_cast<int>(row_pitch(&desc));
  g.W = desc.pack_bits == 4 ? 1 : code_width(g.K);
  g.seed_lo = static_cast<uint32_t>(desc.seed);
  g.seed_hi = static_cast<uint32_t>(desc.seed >> 32);
  for (int c = 0; c < 3; ++c) {
    const uint32_t md = static_cast<uint32_t>(m[c]);
    g.bq[c] = desc.n[c] / md;
    g.br[c] = desc.n[c] % md;
    g.bmag[c] = md == 1 ? 0xFFFFFFFFu
                        : (md <= 1600 ? static_cast<uint32_t>(((1ull << 32) + md - 1) / md) : 0u);
  }
  uint32_t k0 = g.seed_lo, k1 = g.seed_hi;
  for (int r = 0; r < 10; ++r) {
    g.rk[r][0] = k0;
    g.rk[r][1] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return g;
}

// link cells: edge L = floor((1 + h_R)/2) + 1 (two same-colour cells then never
// share a site one writes and the other reads), raised to min_cell; per
// dimension the largest even count <= n/L, or 1.
void layout_of(const smcx_lattice_desc& d, int M, int* L_out, int m[3], bool local = false) {
  const int hR = shell_reach(static_cast<int>(d.kind), M);
  // a trial reads 1 + h_R half units beyond its cell (the partner's
  // neighbours), 1 + 2 h_R under the local-energy model (theirs too)
  int L = local ? (1 + 2 * hR) / 2 + 1 : (1 + hR) / 2 + 1;
  if (static_cast<int>(d.min_cell) > L) L = static_cast<int>(d.min_cell);
  *L_out = L;
  for (int c = 0; c < 3; ++c) {
    int cnt = static_cast<int>(d.n[c]) / L;
    cnt &= ~1;
    if (cnt < 2 || (d.flags & SMCX_SINGLE_CELL)) cnt = 1;
    m[c] = cnt;
  }
}

}  // namespace

Geom smcx_lattice::geom() const { return geom_of(desc, static_cast<int>(M), L, m); }

namespace {

smcx_status cuda_fail(smcx_lattice* lat, cudaError_t e, const char* what) {
  if (lat) lat->sticky = SMCX_ECUDA;
  return fail(SMCX_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define SMCX_CUDA(lat, call)                                 \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail(lat, e_, #call); \
  } while (0)

smcx_status check_handle(smcx_lattice* lat) {
  if (!lat) return fail(SMCX_EINVAL, "null handle");
  if (lat->sticky != SMCX_OK)
    return fail(SMCX_ESTATE, "handle is in an error state from an earlier call");
  return SMCX_OK;
}

ShellParam shell_param(int kind) {
  ShellParam sp;
  std::memset(&sp, 0, sizeof(sp));
  const int total = shell_start(kind, kMaxShells);
  for (int i = 0; i < total; ++i) {
    const ShellVec v = shell_vec(kind, i);
    sp.v[i][0] = v.x;
    sp.v[i][1] = v.y;
    sp.v[i][2] = v.z;
  }
  for (int m = 0; m <= kMaxShells; ++m) sp.start[m] = shell_start(kind, m);
  return sp;
}

void compute_layout(smcx_lattice* lat) {
  layout_of(lat->desc, static_cast<int>(lat->M), &lat->L, lat->m, lat->local);
}

smcx_status validate_occupancy(const smcx_lattice_desc& d, const uint8_t* h) {
  const uint64_t N = n_sites(&d);
  for (uint64_t i = 0; i < N; ++i)
    if (h[i] >= d.n_species) return fail(SMCX_EINVAL, "species id >= n_species in occupancy");
  return SMCX_OK;
}

// The transfer buffer (workspace scratch) is free on the lattice's stream
// once an asynchronous read-back started earlier has copied it out.
smcx_status scratch_guard(smcx_lattice* lat) {
  if (lat->down_pending) SMCX_CUDA(lat, cudaStreamWaitEvent(lat->stream, lat->ev_down, 0));
  return SMCX_OK;
}

// canonical host bytes -> workspace scratch -> (validated on the device) ->
// device storage
smcx_status upload_occupancy(smcx_lattice* lat, const uint8_t* h) {
  if (scratch_guard(lat) != SMCX_OK) return SMCX_ECUDA;
  const Geom g = lat->geom();
  const uint32_t n_cells = static_cast<uint32_t>(lat->N / lat->nb);
  SMCX_CUDA(lat, cudaMemcpyAsync(lat->scratch(), h, lat->N, cudaMemcpyHostToDevice, lat->stream));
  SMCX_CUDA(lat, cudaMemsetAsync(lat->flag(), 0, sizeof(unsigned int), lat->stream));
  SMCX_CUDA(lat, launch_validate(lat->scratch(), lat->N, lat->desc.n_species, lat->flag(),
                                 lat->n_sm, lat->stream));
  // the conversion skips itself when the validation flagged a byte, so an
  // invalid upload leaves the lattice as it was
  SMCX_CUDA(lat, launch_canon_to_dev(g, lat->scratch(), lat->d_occ, n_cells, lat->n_sm,
                                     lat->stream, lat->flag()));
  unsigned int bad = 0;
  SMCX_CUDA(lat, cudaMemcpyAsync(&bad, lat->flag(), sizeof(bad), cudaMemcpyDeviceToHost,
                                 lat->stream));
  SMCX_CUDA(lat, cudaStreamSynchronize(lat->stream));
  if (bad) return fail(SMCX_EINVAL, "species id >= n_species in occupancy");
  return SMCX_OK;
}

smcx_status download_occupancy(smcx_lattice* lat, uint8_t* h) {
  if (scratch_guard(lat) != SMCX_OK) return SMCX_ECUDA;
  const Geom g = lat->geom();
  const uint32_t n_cells = static_cast<uint32_t>(lat->N / lat->nb);
  SMCX_CUDA(lat, launch_dev_to_canon(g, lat->d_occ, lat->scratch(), n_cells, lat->n_sm,
                                     lat->stream));
  SMCX_CUDA(lat, cudaMemcpyAsync(h, lat->scratch(), lat->N, cudaMemcpyDeviceToHost, lat->stream));
  SMCX_CUDA(lat, cudaStreamSynchronize(lat->stream));
  return SMCX_OK;
}

smcx_status run_pair_counts(smcx_lattice* lat, uint32_t n_shells, std::vector<uint64_t>* out) {
  TraceRange trace("smcx_pair_counts");
  const size_t K = lat->desc.n_species;
  const size_t n_cnt = n_shells * K * K;
  Geom g = lat->geom();
  out->assign(n_cnt, 0);
  if (K <= 6) {
    // tiled half-shell counts H (rows of KMAX species); N = H + H^T
    const size_t kmax = K <= 5 ? 5 : 6;
    const int ms = n_shells < 2 ? 2 : static_cast<int>(n_shells);
    const size_t n_h = static_cast<size_t>(ms) * kmax * kmax;
    SMCX_CUDA(lat, cudaMemsetAsync(lat->pairs(), 0, sizeof(uint64_t) * n_h, lat->stream));
    SMCX_CUDA(lat, launch_pair_count_tiled(g, static_cast<int>(n_shells), lat->d_occ, lat->pairs(),
                                           lat->n_sm, lat->stream, false));
    std::vector<uint64_t> h(n_h);
    SMCX_CUDA(lat, cudaMemcpyAsync(h.data(), lat->pairs(), sizeof(uint64_t) * n_h,
                                   cudaMemcpyDeviceToHost, lat->stream));
    SMCX_CUDA(lat, cudaStreamSynchronize(lat->stream));
    for (size_t m = 0; m < n_shells; ++m)
      for (size_t a = 0; a < K; ++a)
        for (size_t b = 0; b < K; ++b)
          (*out)[(m * K + a) * K + b] = h[(m * kmax + a) * kmax + b] + h[(m * kmax + b) * kmax + a];
    return SMCX_OK;
  }
  SMCX_CUDA(lat, cudaMemsetAsync(lat->pairs(), 0, sizeof(uint64_t) * n_cnt, lat->stream));
  const ShellParam sp = shell_param(g.kind);
  SMCX_CUDA(lat, launch_pair_count_generic(g, sp, static_cast<int>(n_shells), lat->d_occ,
                                           lat->pairs(), static_cast<uint32_t>(lat->N / lat->nb),
                                           lat->n_sm, lat->stream));
  SMCX_CUDA(lat, cudaMemcpyAsync(out->data(), lat->pairs(), sizeof(uint64_t) * n_cnt,
                                 cudaMemcpyDeviceToHost, lat->stream));
  SMCX_CUDA(lat, cudaStreamSynchronize(lat->stream));
  return SMCX_OK;
}

// E = 1/2 sum_m sum_{p',p} N_m[p'][p] V_m(p',p): every bond is seen from both
// ends in the directed counts; int128 accumulation.
smcx_status energy_from_counts(smcx_lattice* lat, const std::vector<uint64_t>& cnt, int64_t* e) {
  const size_t K = lat->desc.n_species;
  __int128 acc = 0;
  for (size_t m = 0; m < lat->M; ++m)
    for (size_t a = 0; a < K; ++a)
      for (size_t b = 0; b < K; ++b) {
        const size_t idx = (m * K + a) * K + b;
        acc += static_cast<__int128>(cnt[idx]) * lat->V[idx];
      }
  if (acc % 2 != 0) return fail(SMCX_EINVAL, "internal: odd directed energy");
  acc /= 2;
  if (acc > static_cast<__int128>(INT64_MAX) || acc < static_cast<__int128>(INT64_MIN))
    return fail(SMCX_EOVERFLOW, "energy does not fit int64");
  *e = static_cast<int64_t>(acc);
  return SMCX_OK;
}

// Local-energy model: per-block int64 partial sums of the site energies,
// added on the host in int128.
smcx_status local_energy(smcx_lattice* lat, int64_t* e) {
  const Geom g = lat->geom();
  SMCX_CUDA(lat, launch_local_energy(g, lat->dlp(), lat->dT(), lat->n_T, lat->d_occ, lat->dpart(),
                                     kLocalPartials, lat->stream));
  std::vector<long long> part(kLocalPartials);
  SMCX_CUDA(lat, cudaMemcpyAsync(part.data(), lat->dpart(), sizeof(long long) * kLocalPartials,
                                 cudaMemcpyDeviceToHost, lat->stream));
  SMCX_CUDA(lat, cudaStreamSynchronize(lat->stream));
  __int128 acc = 0;
  for (long long v : part) acc += v;
  if (acc > static_cast<__int128>(INT64_MAX) || acc < static_cast<__int128>(INT64_MIN))
    return fail(SMCX_EOVERFLOW, "energy does not fit int64");
  *e = static_cast<int64_t>(acc);
  return SMCX_OK;
}

smcx_status full_energy(smcx_lattice* lat, int64_t* e) {
  if (lat->local) return local_energy(lat, e);
  std::vector<uint64_t> cnt;
  smcx_status s = run_pair_counts(lat, lat->M, &cnt);
  if (s != SMCX_OK) return s;
  return energy_from_counts(lat, cnt, e);
}

// Restarts the running energy: the accepted-dE sums start again from zero
// and its base E0 is the full energy of the configuration now (one pair
// count, or the local-energy reduction), so that E0 + the sum of accepted dE
// stays an independent check of any later full recompute.  A lattice with no
// model yet takes its base when the model is set.
smcx_status restart_running_energy(smcx_lattice* lat) {
  SMCX_CUDA(lat, cudaMemsetAsync(lat->stats(), 0, sizeof(unsigned long long) * 8, lat->stream));
  lat->e0_known = false;
  if (!lat->has_epi) return SMCX_OK;
  int64_t e = 0;
  const smcx_status s = full_energy(lat, &e);
  if (s != SMCX_OK) return s;
  lat->E0 = e;
  lat->e0_known = true;
  return SMCX_OK;
}

// tile shape the tiled kernel uses (-1 if it cannot run the lattice)
int tiled_shape_for(smcx_lattice* lat) {
  const Geom g = lat->geom();
  if (!lat->tiled_table_ok) return -1;
  if (lat->opt_tile >= 0) return tiled_supported(g, lat->opt_tile) ? lat->opt_tile : -1;
  if (lat->opt_kernel == 0 && lat->tune.done && lat->tune.cands[lat->tune.choice].first == 2)
    return lat->tune.cands[lat->tune.choice].second;
  for (int sh = 0; sh < tiled_shape_count(g.kind); ++sh)
    if (tiled_supported(g, sh)) return sh;
  return -1;
}

bool cell_ok(smcx_lattice* lat) { return lat->tiled_table_ok && cell_supported(lat->geom()); }

// which kernel a colour phase runs: 1 = generic, 2 = tiled, 3 = cell (0 =
// the requested kernel cannot run the lattice).  Automatic: the tuned
// choice, and before tuning has finished tiled, else cell, else generic.
int kernel_choice(smcx_lattice* lat) {
  if (lat->local) return 4;  // the local-energy model has one kernel
  switch (lat->opt_kernel) {
    case 1: return 1;
    case 2: return tiled_shape_for(lat) >= 0 ? 2 : 0;
    case 3: return cell_ok(lat) ? 3 : 0;
    default:
      if (lat->tune.done) return lat->tune.cands[lat->tune.choice].first;
      if (tiled_shape_for(lat) >= 0) return 2;
      return cell_ok(lat) ? 3 : 1;
  }
}

// candidates of the online choice; with fewer than two it is decided at once
void tuning_reset(smcx_lattice* lat) {
  auto& tu = lat->tune;
  tu.done = false;
  tu.cands.clear();
  tu.next = 0;
  tu.choice = 0;
  if (lat->has_epi && lat->tiled_table_ok && !lat->local) {
    const Geom g = lat->geom();
    for (int sh = 0; sh < tiled_shape_count(g.kind); ++sh)
      if (tiled_supported(g, sh)) tu.cands.emplace_back(2, sh);
    if (cell_ok(lat)) tu.cands.emplace_back(3, -1);
  }
  if (lat->local) tu.cands.emplace_back(4, -1);  // the local-energy model's one kernel
  if (tu.cands.empty()) tu.cands.emplace_back(1, -1);
  tu.best_ms.assign(tu.cands.size(), 0.0f);
  tu.samples.assign(tu.cands.size(), 0);
  // nothing to decide with one candidate or a kernel / tile shape forced
  tu.done = tu.cands.size() < 2 || lat->opt_kernel != 0 || lat->opt_tile >= 0;
}

bool colour_empty(smcx_lattice* lat, int colour) {
  for (int d = 0; d < 3; ++d)
    if (lat->m[d] == 1 && ((colour >> d) & 1)) return true;  // no cell of this colour
  return false;
}

// active z cells of a colour whose link-cell z index lies in [c_lo, c_hi):
// indices a in [*az0, *az0 + *naz) of the cells c_z = 2 a + bit
void colour_z_range(const int m[3], int colour, int c_lo, int c_hi, int* az0, int* naz) {
  const int bit = (colour >> 2) & 1;
  if (m[2] == 1) {
    *az0 = 0;
    *naz = (bit == 0 && c_lo <= 0 && c_hi > 0) ? 1 : 0;
    return;
  }
  const int A = m[2] / 2;
  int a0 = (c_lo - bit + 1) >> 1, a1 = (c_hi - bit + 1) >> 1;  // ceil((c - bit) / 2)
  a0 = a0 < 0 ? 0 : a0;
  a1 = a1 > A ? A : a1;
  *az0 = a0;
  *naz = a1 > a0 ? a1 - a0 : 0;
}

// one colour phase of the current sweep with kernel `kern` (tiled: shape),
// over the link cells whose z index lies in [c_lo, c_hi) (c_hi < 0: all)
smcx_status launch_colour_with(smcx_lattice* lat, int colour, const PhaseArgs& base,
                               const Tables& tab, int kern, int shape, int c_lo = 0,
                               int c_hi = -1) {
  TraceRange trace("smcx_colour_phase");
  PhaseArgs a = base;
  a.colour = colour;
  a.staging = lat->opt_staging;
  const Geom g = lat->geom();
  if (colour_empty(lat, colour)) return SMCX_OK;
  colour_z_range(lat->m, colour, c_lo, c_hi < 0 ? lat->m[2] : c_hi, &a.az0, &a.naz);
  if (a.naz == 0) return SMCX_OK;  // no cell of this colour in the range
  if (kern == 0)
    return fail(SMCX_EINVAL, "the requested kernel does not support this lattice/EPI/tile shape");
  if (kern == 4) {
    SMCX_CUDA(lat, launch_sweep_local(g, a, tab, lat->d_occ, lat->dlp(), lat->dT(), lat->n_T,
                                      lat->t32, lat->n_items, lat->stats(), lat->stream));
    return SMCX_OK;
  }
  if (kern == 3) {
    SMCX_CUDA(lat, launch_sweep_cells(g, a, tab, lat->d_occ,
                                      reinterpret_cast<const uint8_t*>(lat->dtab()), lat->stats(),
                                      lat->stream));
    return SMCX_OK;
  }
  if (kern == 2) {
    TiledEpi te;
    te.kmax = lat->tiled_kmax;
    te.d_table = lat->dtab();
    SMCX_CUDA(lat, launch_sweep_tiled(g, a, tab, lat->d_occ, te, lat->stats(), shape, lat->stream));
    return SMCX_OK;
  }
  const ShellParam sp = shell_param(g.kind);
  SMCX_CUDA(lat, launch_sweep_generic(g, a, sp, tab, lat->d_occ, lat->dV(), lat->stats(),
                                      lat->stream));
  return SMCX_OK;
}

// one colour phase of the current sweep with the configured kernel
smcx_status launch_colour(smcx_lattice* lat, int colour, const PhaseArgs& base, const Tables& tab,
                          int c_lo = 0, int c_hi = -1) {
  const int kern = kernel_choice(lat);
  return launch_colour_with(lat, colour, base, tab, kern, kern == 2 ? tiled_shape_for(lat) : -1,
                            c_lo, c_hi);
}

// Difference rows of the tiled and cell kernels, one per species pair (p, q)
// at byte (p * kmax + q) * row_bytes, with D_{m,s} = V_m(q,s) - V_m(p,s) and
// the i-j bond term B = (V_1(q,q) - V_1(p,q)) - (V_1(q,p) - V_1(p,p)):
//   K <= 5 (kmax 5): D'_{m,s} = D_{m,s} - D_{m,4} (D_{m,4} = 0 when K < 5) for
//     s = 0..3, stored per shell m as four words, word t holding byte t of
//     D'_{m,0}, .., D'_{m,3}; then the int64 C = 128 sum_{m,s} D'_{m,s} + B;
//   K = 6 (kmax 6): int32 D'_{m,s} = D_{m,s} - D_{m,0} for s = 1..5, then C = B.
// Returns false when a D' does not fit int32.
bool dtable_of(const smcx_lattice_desc& d, int M, const int64_t* Vt, std::vector<uint8_t>* bytes,
               int* kmax_out) {
  const int K = static_cast<int>(d.n_species);
  if (K > 6 || M < 2) return false;
  const int kmax = K <= 5 ? 5 : 6;
  const int rowb = tiled_row_bytes(M, kmax);
  const int doff = tiled_doff_c(M, kmax);
  bytes->assign(static_cast<size_t>(kmax) * kmax * rowb, 0);
  auto V = [&](int m, int a, int b) { return Vt[(static_cast<size_t>(m) * K + a) * K + b]; };
  for (int p = 0; p < K; ++p)
    for (int q = 0; q < K; ++q) {
      uint8_t* row = bytes->data() + static_cast<size_t>(p * kmax + q) * rowb;
      __int128 C = 0;
      for (int m = 0; m < M; ++m) {
        if (kmax == 5) {
          const int64_t d4 = K == 5 ? V(m, q, 4) - V(m, p, 4) : 0;
          uint32_t w[4] = {0, 0, 0, 0};
          for (int s = 0; s < 4; ++s) {
            const int64_t dp = s < K ? (V(m, q, s) - V(m, p, s)) - d4 : -d4;
            if (dp > INT32_MAX || dp < INT32_MIN) return false;
            const uint32_t u = static_cast<uint32_t>(static_cast<int32_t>(dp));
            for (int t = 0; t < 4; ++t) w[t] |= ((u >> (8 * t)) & 0xFFu) << (8 * s);
            C += static_cast<__int128>(128) * dp;
          }
          std::memcpy(row + 16 * m, w, 16);
        } else {
          const int64_t d0 = V(m, q, 0) - V(m, p, 0);
          for (int s = 1; s < K; ++s) {
            const int64_t dp = (V(m, q, s) - V(m, p, s)) - d0;
            if (dp > INT32_MAX || dp < INT32_MIN) return false;
            const int32_t v32 = static_cast<int32_t>(dp);
            std::memcpy(row + 4 * (m * (kmax - 1) + s - 1), &v32, 4);
          }
        }
      }
      C += (V(0, q, q) - V(0, p, q)) - (V(0, q, p) - V(0, p, p));
      if (C > INT64_MAX || C < INT64_MIN) return false;
      const int64_t c64 = static_cast<int64_t>(C);
      std::memcpy(row + doff, &c64, 8);
    }
  if (kmax_out) *kmax_out = kmax;
  return true;
}

bool build_tiled_table(smcx_lattice* lat, std::vector<uint32_t>* out) {
  std::vector<uint8_t> bytes;
  int kmax = 0;
  if (!dtable_of(lat->desc, static_cast<int>(lat->M), lat->V.data(), &bytes, &kmax)) return false;
  out->assign(bytes.size() / 4, 0u);
  std::memcpy(out->data(), bytes.data(), bytes.size());
  lat->tiled_kmax = kmax;
  return true;
}

smcx_status read_call_stats(smcx_lattice* lat, smcx_sweep_stats* out) {
  unsigned long long h[kStatWait + 1];
  SMCX_CUDA(lat, cudaMemcpyAsync(h, lat->stats() + kStatCall, sizeof(h), cudaMemcpyDeviceToHost,
                                 lat->stream));
  SMCX_CUDA(lat, cudaStreamSynchronize(lat->stream));
  if (h[kStatWait] != 0) {
    SMCX_CUDA(lat, cudaMemsetAsync(lat->stats() + kStatWait, 0, sizeof(unsigned long long),
                                   lat->stream));
    return fail(SMCX_ETIMEOUT, "a staging wait of the tiled sweep gave up");
  }
  out->attempts = h[0];
  out->unlike = h[1];
  out->accepted = h[2];
  out->sum_dE_q = static_cast<int64_t>(h[3]);
  return SMCX_OK;
}

uint32_t crc32(const uint8_t* p, size_t n, uint32_t crc = 0) {
  crc = ~crc;
  for (size_t i = 0; i < n; ++i) {
    crc ^= p[i];
    for (int k = 0; k < 8; ++k) crc = (crc >> 1) ^ (0xEDB88320u & (0u - (crc & 1u)));
  }
  return ~crc;
}

}  // namespace

namespace smcx {
smcx_status batch_fail(smcx_status s, const std::string& msg) { return fail(s, msg); }
bool host_build_tables(double T, Tables* tab, int* mode, int* s) { return build_tables(T, tab, mode, s); }
Geom host_geom(const smcx_lattice_desc& d, int M, const int m[3]) {
  int L = 0, mm[3];
  layout_of(d, M, &L, mm);
  return geom_of(d, M, L, m);
}
void host_layout(const smcx_lattice_desc& d, int M, int* L, int m[3]) { layout_of(d, M, L, m); }
bool host_dtable(const smcx_lattice_desc& d, int M, const int64_t* V, std::vector<uint8_t>* out) {
  return dtable_of(d, M, V, out, nullptr);
}
size_t host_occ_bytes(const smcx_lattice_desc& d) { return occ_bytes(&d); }
void host_sweep_origin(const smcx_lattice_desc& d, uint32_t t, int shift[3]) {
  sweep_origin(d, t, shift);
}
bool host_desc_ok(const smcx_lattice_desc* d, std::string* why) { return desc_ok(d, why); }
}  // namespace smcx

extern "C" {

size_t smcx_occupancy_bytes(const smcx_lattice_desc* desc) {
  std::string why;
  if (!desc_ok(desc, &why)) return 0;
  return occ_bytes(desc);
}

size_t smcx_workspace_bytes(const smcx_lattice_desc* desc) {
  std::string why;
  if (!desc_ok(desc, &why)) return 0;
  return work_layout(desc).total;
}

smcx_status smcx_create_lattice(const smcx_lattice_desc* desc, void* d_occ, void* d_work,
                                const uint8_t* h_init, void* cuda_stream, smcx_lattice** out) {
  std::string why;
  if (!out) return fail(SMCX_EINVAL, "null out pointer");
  *out = nullptr;
  if (!desc_ok(desc, &why)) return fail(SMCX_EINVAL, why);
  if (!d_occ || !d_work || !h_init) return fail(SMCX_EINVAL, "null buffer");
  if (reinterpret_cast<uintptr_t>(d_occ) % 16 != 0 || reinterpret_cast<uintptr_t>(d_work) % 256 != 0)
    return fail(SMCX_EINVAL, "occupancy must be 16-byte and workspace 256-byte aligned");
  smcx_status s = SMCX_OK;
  auto* lat = new smcx_lattice();
  lat->desc = *desc;
  lat->nb = basis_count(static_cast<int>(desc->kind));
  lat->N = n_sites(desc);
  lat->d_occ = static_cast<uint8_t*>(d_occ);
  lat->d_work = static_cast<uint8_t*>(d_work);
  lat->stream = static_cast<cudaStream_t>(cuda_stream);
  lat->wl = work_layout(desc);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&lat->n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    delete lat;
    return fail(SMCX_ECUDA, std::string("device query: ") + cudaGetErrorString(e));
  }
  if (cudaMemsetAsync(lat->stats(), 0, sizeof(unsigned long long) * 16, lat->stream) !=
      cudaSuccess) {
    delete lat;
    return fail(SMCX_ECUDA, "workspace clear failed");
  }
  s = upload_occupancy(lat, h_init);
  if (s == SMCX_OK) s = restart_running_energy(lat);
  if (s != SMCX_OK) {
    delete lat;
    return s;
  }
  *out = lat;
  return SMCX_OK;
}

smcx_status smcx_set_epi(smcx_lattice* lat, uint32_t n_shells, const int64_t* v_q) {
  smcx_status s = check_handle(lat);
  if (s != SMCX_OK) return s;
  if (n_shells < 1 || n_shells > kMaxShells) return fail(SMCX_EINVAL, "n_shells must be 1..4");
  if (!v_q) return fail(SMCX_EINVAL, "null EPI table");
  const size_t K = lat->desc.n_species;
  const int64_t vmax = int64_t(1) << 52;
  for (size_t m = 0; m < n_shells; ++m)
    for (size_t a = 0; a < K; ++a)
      for (size_t b = 0; b < K; ++b) {
        const int64_t v = v_q[(m * K + a) * K + b];
        if (v != v_q[(m * K + b) * K + a]) return fail(SMCX_EINVAL, "EPI table is not symmetric");
        if (v >= vmax || v <= -vmax) return fail(SMCX_EINVAL, "EPI value beyond 2^52 q");
      }
  lat->M = n_shells;
  lat->local = false;
  lat->V.assign(v_q, v_q + n_shells * K * K);
  compute_layout(lat);
  std::vector<int64_t> vpad(kMaxShells * K * K, 0);
  std::copy(lat->V.begin(), lat->V.end(), vpad.begin());
  SMCX_CUDA(lat, cudaMemcpyAsync(lat->dV(), vpad.data(), sizeof(int64_t) * vpad.size(),
                                 cudaMemcpyHostToDevice, lat->stream));
  std::vector<uint32_t> dtab;
  lat->tiled_table_ok = build_tiled_table(lat, &dtab);
  if (lat->tiled_table_ok)
    SMCX_CUDA(lat, cudaMemcpyAsync(lat->dtab(), dtab.data(), sizeof(uint32_t) * dtab.size(),
                                   cudaMemcpyHostToDevice, lat->stream));
  SMCX_CUDA(lat, cudaStreamSynchronize(lat->stream));
  lat->has_epi = true;
  tuning_reset(lat);
  s = restart_running_energy(lat);
  if (s != SMCX_OK) lat->has_epi = false;
  return s;
}

uint32_t smcx_local_model_width(uint32_t kind, uint32_t n_shells) {
  if (kind > 1 || n_shells < 1 || n_shells > static_cast<uint32_t>(kLocalMaxShells)) return 0;
  int z = 0;
  for (uint32_t m = 0; m < n_shells; ++m) z = std::max(z, shell_z(static_cast<int>(kind), m));
  return static_cast<uint32_t>(z + 1);
}

smcx_status smcx_set_local_model(smcx_lattice* lat, uint32_t n_shells, const int64_t* t_q) {
  smcx_status s = check_handle(lat);
  if (s != SMCX_OK) return s;
  const int kind = static_cast<int>(lat->desc.kind);
  const uint32_t zt = smcx_local_model_width(lat->desc.kind, n_shells);
  if (zt == 0) return fail(SMCX_EINVAL, "n_shells must be 1..3 for the local-energy model");
  const size_t K = lat->desc.n_species;
  if (K > static_cast<size_t>(kLocalMaxK)) return fail(SMCX_EINVAL, "local-energy model: K <= 8");
  if (!t_q) return fail(SMCX_EINVAL, "null table");
  for (int d = 0; d < 3; ++d)
    if (lat->desc.n[d] < 4) return fail(SMCX_EINVAL, "local-energy model: every n_d >= 4");
  const size_t n_T = static_cast<size_t>(n_shells) * K * K * zt;
  for (size_t i = 0; i < n_T; ++i)
    if (t_q[i] > kLocalMaxAbsT || t_q[i] < -kLocalMaxAbsT)
      return fail(SMCX_EINVAL, "local-energy table value beyond 2^48 q");
  LocalParam lp;
  std::memset(&lp, 0, sizeof(lp));
  lp.M = static_cast<int>(n_shells);
  lp.K = static_cast<int>(K);
  lp.zt = static_cast<int>(zt);
  lp.total = shell_start(kind, lp.M);
  for (int m = 0; m <= lp.M; ++m) lp.start[m] = shell_start(kind, m);
  for (int t = 0; t < lp.total; ++t) {
    const ShellVec v = shell_vec(kind, t);
    lp.v[t][0] = static_cast<int8_t>(v.x);
    lp.v[t][1] = static_cast<int8_t>(v.y);
    lp.v[t][2] = static_cast<int8_t>(v.z);
  }
  // U as distinct displacements from i: 0, the partner d, the shell vectors,
  // and d plus each shell vector
  const int z1 = shell_z(kind, 0);
  for (int dir = 0; dir < z1; ++dir) {
    const ShellVec d = shell_vec(kind, dir);
    std::vector<std::array<int, 3>> u;
    auto add = [&](int x, int y, int z) {
      for (const auto& e : u)
        if (e[0] == x && e[1] == y && e[2] == z) return;
      u.push_back({x, y, z});
    };
    add(0, 0, 0);
    add(d.x, d.y, d.z);
    for (int t = 0; t < lp.total; ++t) {
      const ShellVec v = shell_vec(kind, t);
      add(v.x, v.y, v.z);
    }
    for (int t = 0; t < lp.total; ++t) {
      const ShellVec v = shell_vec(kind, t);
      add(d.x + v.x, d.y + v.y, d.z + v.z);
    }
    lp.n_u[dir] = static_cast<int>(u.size());
    for (size_t e = 0; e < u.size(); ++e) {
      for (int c = 0; c < 3; ++c) lp.u[dir][e][c] = static_cast<int8_t>(u[e][c]);
      // shells of site k = i + u holding i (vector -u) and j (vector d - u);
      // with n_d >= 4 no two of these displacements name the same site
      for (int m = 0; m < lp.M; ++m)
        for (int t = shell_start(kind, m); t < shell_start(kind, m + 1); ++t) {
          const ShellVec v = shell_vec(kind, t);
          if (v.x == -u[e][0] && v.y == -u[e][1] && v.z == -u[e][2])
            lp.shells_i[dir][e] |= static_cast<uint8_t>(1u << m);
          if (v.x == d.x - u[e][0] && v.y == d.y - u[e][1] && v.z == d.z - u[e][2])
            lp.shells_j[dir][e] |= static_cast<uint8_t>(1u << m);
        }
    }
  }
  // the items: (e, m) with exactly one of i, j in shell m+1 of site e, by shell
  for (int dir = 0; dir < z1; ++dir) {
    int n = 0;
    for (int m = 0; m < lp.M; ++m)
      for (int e = 2; e < lp.n_u[dir]; ++e) {
        const uint32_t mi = (lp.shells_i[dir][e] >> m) & 1u, mj = (lp.shells_j[dir][e] >> m) & 1u;
        if (mi == mj) continue;
        if (n >= kLocalMaxItems) return fail(SMCX_EINVAL, "internal: local item list overflow");
        lp.item_e[dir][n] = static_cast<uint8_t>(e);
        lp.item_m[dir][n] = static_cast<uint8_t>(m | (mj << 2));
        ++n;
      }
    if (dir == 0) lp.n_items = n;
    if (n != lp.n_items) return fail(SMCX_EINVAL, "internal: directions differ in item count");
    for (int x = 0; x < n; ++x)
      if ((lp.item_m[dir][x] & 3) != (lp.item_m[0][x] & 3))
        return fail(SMCX_EINVAL, "internal: directions differ in item shells");
  }
  SMCX_CUDA(lat, cudaMemcpyAsync(lat->dlp(), &lp, sizeof(lp), cudaMemcpyHostToDevice, lat->stream));
  SMCX_CUDA(lat, cudaMemcpyAsync(lat->dT(), t_q, sizeof(int64_t) * n_T, cudaMemcpyHostToDevice,
                                 lat->stream));
  SMCX_CUDA(lat, cudaStreamSynchronize(lat->stream));
  lat->M = n_shells;
  lat->local = true;
  lat->zt = static_cast<int>(zt);
  lat->n_T = static_cast<int>(n_T);
  lat->n_items = lp.n_items;
  lat->t32 = true;
  for (size_t i = 0; i < n_T; ++i)
    lat->t32 = lat->t32 && t_q[i] >= INT32_MIN && t_q[i] <= INT32_MAX;
  lat->V.clear();
  lat->tiled_table_ok = false;
  lat->has_epi = true;
  compute_layout(lat);
  tuning_reset(lat);
  return restart_running_energy(lat);
}

constexpr int kTuneSamples = 3;  // timed phases per candidate

smcx_status smcx_sweep(smcx_lattice* lat, uint32_t n_sweeps, double T_first, double T_last,
                       smcx_sweep_stats* out) {
  TraceRange trace("smcx_sweep");
  smcx_status s = check_handle(lat);
  if (s != SMCX_OK) return s;
  if (!lat->has_epi) return fail(SMCX_ESTATE, "set_epi must be called before sweep");
  if (std::isnan(T_first) || std::isnan(T_last) || T_first < 0 || T_last < 0)
    return fail(SMCX_EINVAL, "temperatures must be >= 0");
  SMCX_CUDA(lat, cudaMemsetAsync(lat->stats() + kStatCall, 0, sizeof(unsigned long long) * 4,
                                 lat->stream));
  // online kernel choice: while untuned, phases rotate over the candidates
  // and are timed with events (every candidate gives the same bits)
  auto& tu = lat->tune;
  const bool tuning = lat->opt_kernel == 0 && lat->opt_tile < 0 && !tu.done;
  const size_t max_timed = tuning ? tu.cands.size() * kTuneSamples : 0;
  std::vector<int> timed;  // candidate of each timed phase
  while (tu.ev.size() < 2 * max_timed) {
    cudaEvent_t e;
    SMCX_CUDA(lat, cudaEventCreate(&e));
    tu.ev.push_back(e);
  }
  Tables tab;
  for (uint32_t i = 0; i < n_sweeps; ++i) {
    double T = T_first;
    if (n_sweeps > 1 && T_first != T_last)
      T = T_first + (T_last - T_first) * static_cast<double>(i) / static_cast<double>(n_sweeps - 1);
    PhaseArgs a{};
    if (!build_tables(T, &tab, &a.mode, &a.s)) return fail(SMCX_EINVAL, "bad temperature");
    a.t = lat->t;
    sweep_origin(lat->desc, a.t, a.shift);
    for (int colour = 0; colour < 8; ++colour) {
      if (tuning && timed.size() < max_timed && !colour_empty(lat, colour)) {
        const int c = static_cast<int>(tu.next++ % tu.cands.size());
        const size_t k = timed.size();
        SMCX_CUDA(lat, cudaEventRecord(tu.ev[2 * k], lat->stream));
        s = launch_colour_with(lat, colour, a, tab, tu.cands[c].first, tu.cands[c].second);
        if (s != SMCX_OK) return s;
        SMCX_CUDA(lat, cudaEventRecord(tu.ev[2 * k + 1], lat->stream));
        timed.push_back(c);
        continue;
      }
      s = launch_colour(lat, colour, a, tab);
      if (s != SMCX_OK) return s;
    }
    lat->t += 1;
  }
  if (!timed.empty()) {
    SMCX_CUDA(lat, cudaEventSynchronize(tu.ev[2 * timed.size() - 1]));
    for (size_t k = 0; k < timed.size(); ++k) {
      float ms = 0;
      SMCX_CUDA(lat, cudaEventElapsedTime(&ms, tu.ev[2 * k], tu.ev[2 * k + 1]));
      const int c = timed[k];
      if (tu.samples[c] == 0 || ms < tu.best_ms[c]) tu.best_ms[c] = ms;
      ++tu.samples[c];
    }
    bool all = true;
    for (int n : tu.samples) all = all && n >= kTuneSamples;
    if (all) {
      int best = 0;
      for (size_t c = 1; c < tu.cands.size(); ++c)
        if (tu.best_ms[c] < tu.best_ms[best]) best = static_cast<int>(c);
      tu.choice = best;
      tu.done = true;
    }
  }
  if (out) return read_call_stats(lat, out);
  return SMCX_OK;
}

smcx_status smcx_run_colour(smcx_lattice* lat, uint32_t colour, double T, smcx_sweep_stats* out) {
  smcx_status s = check_handle(lat);
  if (s != SMCX_OK) return s;
  if (!lat->has_epi) return fail(SMCX_ESTATE, "set_epi must be called before run_colour");
  if (colour > 7) return fail(SMCX_EINVAL, "colour must be 0..7");
  Tables tab;
  PhaseArgs a{};
  if (!build_tables(T, &tab, &a.mode, &a.s)) return fail(SMCX_EINVAL, "temperature must be >= 0");
  SMCX_CUDA(lat, cudaMemsetAsync(lat->stats() + kStatCall, 0, sizeof(unsigned long long) * 4,
                                 lat->stream));
  a.t = lat->t;
  sweep_origin(lat->desc, a.t, a.shift);
  s = launch_colour(lat, static_cast<int>(colour), a, tab);
  if (s != SMCX_OK) return s;
  if (out) return read_call_stats(lat, out);
  return SMCX_OK;
}

smcx_status smcx_run_colour_planes(smcx_lattice* lat, uint32_t colour, double T, int32_t c_lo,
                                   int32_t c_hi, smcx_sweep_stats* out) {
  smcx_status s = check_handle(lat);
  if (s != SMCX_OK) return s;
  if (!lat->has_epi) return fail(SMCX_ESTATE, "set_epi must be called before run_colour_planes");
  if (colour > 7) return fail(SMCX_EINVAL, "colour must be 0..7");
  if (c_lo < 0 || c_hi < c_lo || c_hi > lat->m[2])
    return fail(SMCX_EINVAL, "need 0 <= c_lo <= c_hi <= m_z");
  Tables tab;
  PhaseArgs a{};
  if (!build_tables(T, &tab, &a.mode, &a.s)) return fail(SMCX_EINVAL, "temperature must be >= 0");
  SMCX_CUDA(lat, cudaMemsetAsync(lat->stats() + kStatCall, 0, sizeof(unsigned long long) * 4,
                                 lat->stream));
  a.t = lat->t;
  sweep_origin(lat->desc, a.t, a.shift);
  if (c_hi > c_lo) {
    s = launch_colour(lat, static_cast<int>(colour), a, tab, c_lo, c_hi);
    if (s != SMCX_OK) return s;
  }
  if (out) return read_call_stats(lat, out);
  return SMCX_OK;
}

size_t smcx_planes_bytes(smcx_lattice* lat, uint32_t nz) {
  if (!lat) return 0;
  const size_t groups = lat->desc.pack_bits == 4 ? lat->nb / 2 : lat->nb;
  return groups * nz * lat->desc.n[1] * row_pitch(&lat->desc);
}

}  // extern "C"

namespace {
// the runs of planes z0 .. z0 + nz - 1 (mod n_z) in each row group: calls
// f(group, first plane, planes, offset of the run in the packed buffer)
template <class F>
smcx_status for_plane_runs(smcx_lattice* lat, int32_t z0, uint32_t nz, const void* buf, F f) {
  const int n_z = static_cast<int>(lat->desc.n[2]);
  if (z0 < 0 || z0 >= n_z || nz == 0 || nz > static_cast<uint32_t>(n_z))
    return fail(SMCX_EINVAL, "planes: need 0 <= z0 < n_z and 1 <= nz <= n_z");
  if (!buf || reinterpret_cast<uintptr_t>(buf) % 16 != 0)
    return fail(SMCX_EINVAL, "planes: null or not 16-byte aligned buffer");
  const size_t groups = lat->desc.pack_bits == 4 ? lat->nb / 2 : lat->nb;
  const size_t plane = static_cast<size_t>(lat->desc.n[1]) * row_pitch(&lat->desc);
  const int first = static_cast<int>(nz) < n_z - z0 ? static_cast<int>(nz) : n_z - z0;
  for (size_t g = 0; g < groups; ++g) {
    const size_t base = g * nz * plane;
    smcx_status s = f(g, z0, first, base);
    if (s == SMCX_OK && first < static_cast<int>(nz))
      s = f(g, 0, static_cast<int>(nz) - first, base + first * plane);
    if (s != SMCX_OK) return s;
  }
  return SMCX_OK;
}

size_t plane_bytes(smcx_lattice* lat) {
  return static_cast<size_t>(lat->desc.n[1]) * row_pitch(&lat->desc);
}

uint8_t* plane_ptr(smcx_lattice* lat, size_t g, int z) {
  return lat->d_occ + (g * lat->desc.n[2] + static_cast<size_t>(z)) * plane_bytes(lat);
}
}  // namespace

extern "C" {

smcx_status smcx_get_planes(smcx_lattice* lat, int32_t z0, uint32_t nz, void* d_dst) {
  smcx_status s = check_handle(lat);
  if (s != SMCX_OK) return s;
  uint8_t* dst = static_cast<uint8_t*>(d_dst);
  return for_plane_runs(lat, z0, nz, d_dst, [&](size_t g, int z, int k, size_t off) {
    SMCX_CUDA(lat, cudaMemcpyAsync(dst + off, plane_ptr(lat, g, z), k * plane_bytes(lat),
                                   cudaMemcpyDeviceToDevice, lat->stream));
    return SMCX_OK;
  });
}

smcx_status smcx_put_planes(smcx_lattice* lat, int32_t z0, uint32_t nz, const void* d_src) {
  smcx_status s = check_handle(lat);
  if (s != SMCX_OK) return s;
  const uint8_t* src = static_cast<const uint8_t*>(d_src);
  return for_plane_runs(lat, z0, nz, d_src, [&](size_t g, int z, int k, size_t off) {
    SMCX_CUDA(lat, cudaMemcpyAsync(plane_ptr(lat, g, z), src + off, k * plane_bytes(lat),
                                   cudaMemcpyDeviceToDevice, lat->stream));
    return SMCX_OK;
  });
}

smcx_status smcx_merge_planes(smcx_lattice* lat, int32_t z0, uint32_t nz, const void* d_theirs,
                              const void* d_before) {
  smcx_status s = check_handle(lat);
  if (s != SMCX_OK) return s;
  if (!d_before || reinterpret_cast<uintptr_t>(d_before) % 16 != 0)
    return fail(SMCX_EINVAL, "planes: null or not 16-byte aligned buffer");
  const uint8_t* th = static_cast<const uint8_t*>(d_theirs);
  const uint8_t* bf = static_cast<const uint8_t*>(d_before);
  return for_plane_runs(lat, z0, nz, d_theirs, [&](size_t g, int z, int k, size_t off) {
    SMCX_CUDA(lat, launch_merge_planes(plane_ptr(lat, g, z), th + off, bf + off,
                                       k * plane_bytes(lat), lat->n_sm, lat->stream));
    return SMCX_OK;
  });
}

smcx_status smcx_energy(smcx_lattice* lat, int64_t* e_q) {
  smcx_status s = check_handle(lat);
  if (s != SMCX_OK) return s;
  if (!lat->has_epi) return fail(SMCX_ESTATE, "no EPI set");
  if (!e_q) return fail(SMCX_EINVAL, "null output");
  return full_energy(lat, e_q);
}

smcx_status smcx_running_energy(smcx_lattice* lat, int64_t* e_q) {
  smcx_status s = check_handle(lat);
  if (s != SMCX_OK) return s;
  if (!lat->has_epi) return fail(SMCX_ESTATE, "no EPI set");
  if (!e_q) return fail(SMCX_EINVAL, "null output");
  if (!lat->e0_known) return fail(SMCX_ESTATE, "running energy has no base");
  unsigned long long cum_de = 0;
  SMCX_CUDA(lat, cudaMemcpyAsync(&cum_de, lat->stats() + kStatCum + 3, sizeof(cum_de),
                                 cudaMemcpyDeviceToHost, lat->stream));
  SMCX_CUDA(lat, cudaStreamSynchronize(lat->stream));
  *e_q = static_cast<int64_t>(static_cast<uint64_t>(lat->E0) + cum_de);
  return SMCX_OK;
}

smcx_status smcx_warren_cowley_sro(smcx_lattice* lat, uint32_t n_shells, uint64_t* pair_counts,
                                   double* alpha) {
  smcx_status s = check_handle(lat);
  if (s != SMCX_OK) return s;
  if (n_shells < 1 || n_shells > kMaxShells) return fail(SMCX_EINVAL, "n_shells must be 1..4");
  if (!pair_counts) return fail(SMCX_EINVAL, "null pair_counts");
  std::vector<uint64_t> cnt;
  s = run_pair_counts(lat, n_shells, &cnt);
  if (s != SMCX_OK) return s;
  std::memcpy(pair_counts, cnt.data(), sizeof(uint64_t) * cnt.size());
  if (!alpha) return SMCX_OK;
  const size_t K = lat->desc.n_species;
  // species totals: N_p = sum over centres of shell-1 counts / z_1
  std::vector<uint64_t> Np(K, 0);
  const uint64_t z1 = static_cast<uint64_t>(shell_z(static_cast<int>(lat->desc.kind), 0));
  for (size_t a = 0; a < K; ++a) {
    uint64_t row = 0;
    for (size_t b = 0; b < K; ++b) row += cnt[a * K + b];
    Np[a] = row / z1;
  }
  const double N = static_cast<double>(lat->N);
  for (size_t m = 0; m < n_shells; ++m) {
    const double zm = static_cast<double>(shell_z(static_cast<int>(lat->desc.kind), static_cast<int>(m)));
    for (size_t pc = 0; pc < K; ++pc)
      for (size_t p = 0; p < K; ++p) {
        const double n_centre = static_cast<double>(Np[pc]);
        const double n_p = static_cast<double>(Np[p]);
        const double cond = static_cast<double>(cnt[(m * K + pc) * K + p]) / (n_centre * zm);
        const double conc = n_p / N;
        alpha[(m * K + pc) * K + p] = (n_centre > 0 && n_p > 0) ? 1.0 - cond / conc : NAN;
      }
  }
  return SMCX_OK;
}

smcx_status smcx_composition_profile(smcx_lattice* lat, uint32_t axis, const int32_t* origin_h,
                                     uint64_t radius2_h, uint32_t length_h, uint32_t n_bins,
                                     uint64_t* counts) {
  TraceRange trace("smcx_composition_profile");
  smcx_status s = check_handle(lat);
  if (s != SMCX_OK) return s;
  if (axis > 2 || !origin_h || !counts) return fail(SMCX_EINVAL, "bad axis or null argument");
  const uint64_t K = lat->desc.n_species;
  if (n_bins < 1 || length_h < 1 || length_h > 2 * lat->desc.n[axis])
    return fail(SMCX_EINVAL, "need n_bins >= 1 and 1 <= length_h <= 2 n[axis]");
  if (n_bins * K > 8192 || 8 * n_bins * K > lat->N)
    return fail(SMCX_EINVAL, "too many bins (n_bins * K <= 8192 and 8 n_bins K <= sites)");
  if (scratch_guard(lat) != SMCX_OK) return SMCX_ECUDA;
  const Geom g = lat->geom();
  auto* d_cnt = reinterpret_cast<unsigned long long*>(lat->scratch());
  const size_t bytes = sizeof(uint64_t) * n_bins * K;
  SMCX_CUDA(lat, cudaMemsetAsync(d_cnt, 0, bytes, lat->stream));
  const int o[3] = {origin_h[0], origin_h[1], origin_h[2]};
  SMCX_CUDA(lat, launch_profile(g, lat->d_occ, static_cast<int>(axis), o, radius2_h, length_h, n_bins,
                                d_cnt, lat->n_sm, lat->stream));
  SMCX_CUDA(lat, cudaMemcpyAsync(counts, d_cnt, bytes, cudaMemcpyDeviceToHost, lat->stream));
  SMCX_CUDA(lat, cudaStreamSynchronize(lat->stream));
  return SMCX_OK;
}

smcx_status smcx_clusters(smcx_lattice* lat, uint32_t species_mask, void* d_scratch,
                          size_t scratch_bytes, uint64_t* n_clusters, uint64_t* sizes,
                          uint64_t cap) {
  TraceRange trace("smcx_clusters");
  smcx_status s = check_handle(lat);
  if (s != SMCX_OK) return s;
  if (!n_clusters || (cap && !sizes)) return fail(SMCX_EINVAL, "null output");
  if (!d_scratch || scratch_bytes < 8 * lat->N || reinterpret_cast<uintptr_t>(d_scratch) % 16)
    return fail(SMCX_EINVAL, "scratch must be >= 8 bytes per site and 16-byte aligned");
  if (lat->N >= 0xFFFFFFFFull) return fail(SMCX_EINVAL, "too many sites for 32-bit labels");
  const Geom g = lat->geom();
  auto* lab = static_cast<uint32_t*>(d_scratch);
  uint32_t* cnt = lab + lat->N;
  auto* n_out = reinterpret_cast<unsigned long long*>(lat->pairs());
  auto* err = reinterpret_cast<unsigned int*>(lat->pairs() + 1);
  SMCX_CUDA(lat, cudaMemsetAsync(lat->pairs(), 0, 16, lat->stream));
  SMCX_CUDA(lat, launch_clusters(g, lat->d_occ, species_mask, lab, cnt, n_out, err,
                                 static_cast<uint32_t>(lat->N), lat->n_sm, lat->stream));
  unsigned long long hdr[2] = {0, 0};
  SMCX_CUDA(lat, cudaMemcpyAsync(hdr, lat->pairs(), 16, cudaMemcpyDeviceToHost, lat->stream));
  SMCX_CUDA(lat, cudaStreamSynchronize(lat->stream));
  if (static_cast<unsigned int>(hdr[1]) != 0) {
    lat->sticky = SMCX_ETIMEOUT;
    return fail(SMCX_ETIMEOUT, "cluster labelling: a capped loop gave up");
  }
  *n_clusters = hdr[0];
  if (cap == 0 || hdr[0] == 0) return SMCX_OK;
  std::vector<uint32_t> all(hdr[0]);
  SMCX_CUDA(lat, cudaMemcpyAsync(all.data(), lab, sizeof(uint32_t) * all.size(),
                                 cudaMemcpyDeviceToHost, lat->stream));
  SMCX_CUDA(lat, cudaStreamSynchronize(lat->stream));
  // only the largest `cap` sizes are returned, in descending order
  const size_t top = static_cast<size_t>(std::min<uint64_t>(cap, all.size()));
  std::partial_sort(all.begin(), all.begin() + top, all.end(),
                    [](uint32_t a, uint32_t b) { return a > b; });
  for (size_t k = 0; k < top; ++k) sizes[k] = all[k];
  return SMCX_OK;
}

smcx_status smcx_get_occupancy(smcx_lattice* lat, uint8_t* h_out) {
  smcx_status s = check_handle(lat);
  if (s != SMCX_OK) return s;
  if (!h_out) return fail(SMCX_EINVAL, "null output");
  return download_occupancy(lat, h_out);
}

smcx_status smcx_get_occupancy_async(smcx_lattice* lat, uint8_t* h_out) {
  smcx_status s = check_handle(lat);
  if (s != SMCX_OK) return s;
  if (!h_out) return fail(SMCX_EINVAL, "null output");
  if (!lat->copy) {
    SMCX_CUDA(lat, cudaStreamCreateWithFlags(&lat->copy, cudaStreamNonBlocking));
    SMCX_CUDA(lat, cudaEventCreateWithFlags(&lat->ev_conv, cudaEventDisableTiming));
    SMCX_CUDA(lat, cudaEventCreateWithFlags(&lat->ev_down, cudaEventDisableTiming));
  }
  if (scratch_guard(lat) != SMCX_OK) return SMCX_ECUDA;
  const Geom g = lat->geom();
  SMCX_CUDA(lat, launch_dev_to_canon(g, lat->d_occ, lat->scratch(),
                                     static_cast<uint32_t>(lat->N / lat->nb), lat->n_sm,
                                     lat->stream));
  SMCX_CUDA(lat, cudaEventRecord(lat->ev_conv, lat->stream));
  SMCX_CUDA(lat, cudaStreamWaitEvent(lat->copy, lat->ev_conv, 0));
  SMCX_CUDA(lat, cudaMemcpyAsync(h_out, lat->scratch(), lat->N, cudaMemcpyDeviceToHost,
                                 lat->copy));
  SMCX_CUDA(lat, cudaEventRecord(lat->ev_down, lat->copy));
  lat->down_pending = true;
  return SMCX_OK;
}

smcx_status smcx_wait_occupancy(smcx_lattice* lat) {
  if (!lat) return fail(SMCX_EINVAL, "null handle");
  if (!lat->down_pending) return SMCX_OK;
  SMCX_CUDA(lat, cudaEventSynchronize(lat->ev_down));
  lat->down_pending = false;
  return SMCX_OK;
}

smcx_status smcx_set_occupancy(smcx_lattice* lat, const uint8_t* h_in) {
  smcx_status s = check_handle(lat);
  if (s != SMCX_OK) return s;
  if (!h_in) return fail(SMCX_EINVAL, "null input");
  s = upload_occupancy(lat, h_in);
  if (s != SMCX_OK) return s;
  return restart_running_energy(lat);
}

smcx_status smcx_get_sweep_counter(smcx_lattice* lat, uint32_t* t) {
  if (!lat || !t) return fail(SMCX_EINVAL, "null argument");
  *t = lat->t;
  return SMCX_OK;
}

smcx_status smcx_set_sweep_counter(smcx_lattice* lat, uint32_t t) {
  smcx_status s = check_handle(lat);
  if (s != SMCX_OK) return s;
  lat->t = t;
  return SMCX_OK;
}

smcx_status smcx_get_layout(smcx_lattice* lat, uint32_t* L, uint32_t* m) {
  if (!lat || !L || !m) return fail(SMCX_EINVAL, "null argument");
  if (!lat->has_epi) return fail(SMCX_ESTATE, "layout is fixed by set_epi");
  *L = static_cast<uint32_t>(lat->L);
  for (int c = 0; c < 3; ++c) m[c] = static_cast<uint32_t>(lat->m[c]);
  return SMCX_OK;
}

// checkpoint format (little endian):
//   "SMCXCKP1" | desc (40 bytes) | M u32 | t u32 | E_run i64 | V [M][K][K] i64 |
//   occupancy N bytes | CRC-32 of everything before it (u32)
smcx_status smcx_checkpoint(smcx_lattice* lat, void* buf, size_t* len) {
  smcx_status s = check_handle(lat);
  if (s != SMCX_OK) return s;
  if (!len) return fail(SMCX_EINVAL, "null len");
  if (lat->local) return fail(SMCX_ESTATE, "checkpoints hold EPI lattices only");
  const size_t K = lat->desc.n_species;
  const size_t need = 8 + sizeof(smcx_lattice_desc) + 4 + 4 + 8 + sizeof(int64_t) * lat->M * K * K +
                      lat->N + 4;
  if (!buf) {
    *len = need;
    return SMCX_OK;
  }
  if (*len < need) return fail(SMCX_ENOMEM, "checkpoint buffer too small");
  int64_t e_run = 0;
  if (lat->has_epi) {
    s = smcx_running_energy(lat, &e_run);
    if (s != SMCX_OK) return s;
  }
  uint8_t* p = static_cast<uint8_t*>(buf);
  std::memcpy(p, "SMCXCKP1", 8);
  size_t off = 8;
  std::memcpy(p + off, &lat->desc, sizeof(smcx_lattice_desc));
  off += sizeof(smcx_lattice_desc);
  const uint32_t M = lat->has_epi ? lat->M : 0;
  std::memcpy(p + off, &M, 4);
  off += 4;
  std::memcpy(p + off, &lat->t, 4);
  off += 4;
  std::memcpy(p + off, &e_run, 8);
  off += 8;
  if (M) std::memcpy(p + off, lat->V.data(), sizeof(int64_t) * M * K * K);
  off += sizeof(int64_t) * M * K * K;
  s = download_occupancy(lat, p + off);
  if (s != SMCX_OK) return s;
  off += lat->N;
  const uint32_t crc = crc32(p, off);
  std::memcpy(p + off, &crc, 4);
  off += 4;
  *len = off;
  return SMCX_OK;
}

smcx_status smcx_restore(smcx_lattice* lat, const void* buf, size_t len) {
  smcx_status s = check_handle(lat);
  if (s != SMCX_OK) return s;
  if (!buf) return fail(SMCX_EINVAL, "null buffer");
  const uint8_t* p = static_cast<const uint8_t*>(buf);
  const size_t head = 8 + sizeof(smcx_lattice_desc) + 16;
  if (len < head + 4 || std::memcmp(p, "SMCXCKP1", 8) != 0)
    return fail(SMCX_EINVAL, "not a checkpoint");
  smcx_lattice_desc d;
  std::memcpy(&d, p + 8, sizeof(d));
  if (std::memcmp(&d, &lat->desc, sizeof(d)) != 0)
    return fail(SMCX_EINVAL, "checkpoint was written for another lattice descriptor");
  uint32_t M, t;
  int64_t e_run;
  size_t off = 8 + sizeof(d);
  std::memcpy(&M, p + off, 4);
  std::memcpy(&t, p + off + 4, 4);
  std::memcpy(&e_run, p + off + 8, 8);
  off += 16;
  const size_t K = d.n_species;
  if (M > kMaxShells) return fail(SMCX_EINVAL, "bad shell count in checkpoint");
  const size_t need = off + sizeof(int64_t) * M * K * K + lat->N + 4;
  if (len != need) return fail(SMCX_EINVAL, "checkpoint size mismatch");
  uint32_t crc;
  std::memcpy(&crc, p + need - 4, 4);
  if (crc != crc32(p, need - 4)) return fail(SMCX_EINVAL, "checkpoint CRC mismatch");
  const uint8_t* occ = p + off + sizeof(int64_t) * M * K * K;
  s = validate_occupancy(lat->desc, occ);
  if (s != SMCX_OK) return s;
  if (M) {
    std::vector<int64_t> V(M * K * K);
    std::memcpy(V.data(), p + off, sizeof(int64_t) * V.size());
    s = smcx_set_epi(lat, M, V.data());
    if (s != SMCX_OK) return s;
  }
  s = upload_occupancy(lat, occ);
  if (s != SMCX_OK) return s;
  SMCX_CUDA(lat, cudaMemsetAsync(lat->stats(), 0, sizeof(unsigned long long) * 8, lat->stream));
  SMCX_CUDA(lat, cudaStreamSynchronize(lat->stream));
  lat->E0 = e_run;
  lat->e0_known = true;
  lat->t = t;
  return SMCX_OK;
}

smcx_status smcx_set_option(smcx_lattice* lat, uint32_t key, int64_t value) {
  if (!lat) return fail(SMCX_EINVAL, "null handle");
  if (key == SMCX_OPT_KERNEL) {
    if (value < 0 || value > 3) return fail(SMCX_EINVAL, "kernel option must be 0..3");
    lat->opt_kernel = static_cast<int>(value);
    tuning_reset(lat);
    return SMCX_OK;
  }
  if (key == SMCX_OPT_TILE) {
    if (value < -1 || value >= static_cast<int64_t>(smcx_tile_shape_count(lat->desc.kind)))
      return fail(SMCX_EINVAL, "tile shape index out of range");
    lat->opt_tile = static_cast<int>(value);
    tuning_reset(lat);
    return SMCX_OK;
  }
  if (key == SMCX_OPT_STAGING) {
    if (value < 0 || value > 1) return fail(SMCX_EINVAL, "staging option must be 0 or 1");
    lat->opt_staging = static_cast<int>(value);
    tuning_reset(lat);
    return SMCX_OK;
  }
  return fail(SMCX_EINVAL, "unknown option");
}

uint32_t smcx_tile_shape_count(uint32_t kind) {
  if (kind > 1) return 0;
  return static_cast<uint32_t>(tiled_shape_count(static_cast<int>(kind)));
}

smcx_status smcx_tile_shape(uint32_t kind, uint32_t i, uint32_t* cells_xyz) {
  if (kind > 1 || !cells_xyz || i >= smcx_tile_shape_count(kind))
    return fail(SMCX_EINVAL, "bad tile shape request");
  int c[3];
  tiled_shape_cells(static_cast<int>(kind), static_cast<int>(i), c);
  for (int d = 0; d < 3; ++d) cells_xyz[d] = static_cast<uint32_t>(c[d]);
  return SMCX_OK;
}

smcx_status smcx_kernel_in_use(smcx_lattice* lat, uint32_t* kernel, int32_t* tile_shape) {
  if (!lat || !kernel || !tile_shape) return fail(SMCX_EINVAL, "null argument");
  if (!lat->has_epi) return fail(SMCX_ESTATE, "no EPI set");
  *kernel = static_cast<uint32_t>(kernel_choice(lat));
  *tile_shape = *kernel == 2 ? tiled_shape_for(lat) : -1;
  return SMCX_OK;
}

smcx_status smcx_kernel_tuning(smcx_lattice* lat, uint32_t* done, uint32_t* n_candidates,
                               uint32_t* kernels, int32_t* shapes, float* best_ms) {
  if (!lat || !done || !n_candidates) return fail(SMCX_EINVAL, "null argument");
  if (!lat->has_epi) return fail(SMCX_ESTATE, "no EPI set");
  const auto& tu = lat->tune;
  *done = tu.done ? 1u : 0u;
  const uint32_t cap = *n_candidates;
  *n_candidates = static_cast<uint32_t>(tu.cands.size());
  for (uint32_t c = 0; c < cap && c < tu.cands.size(); ++c) {
    if (kernels) kernels[c] = static_cast<uint32_t>(tu.cands[c].first);
    if (shapes) shapes[c] = tu.cands[c].second;
    if (best_ms) best_ms[c] = tu.samples[c] ? tu.best_ms[c] : -1.0f;
  }
  return SMCX_OK;
}

smcx_status smcx_destroy(smcx_lattice* lat) {
  if (!lat) return fail(SMCX_EINVAL, "null handle");
  delete lat;
  return SMCX_OK;
}

const char* smcx_last_error(void) { return g_err.c_str(); }

uint32_t smcx_shell_table(uint32_t kind, uint32_t n_shells, int32_t* disp, uint32_t cap,
                          uint32_t* z) {
  if (kind > 1 || n_shells < 1 || n_shells > kMaxShells || !disp || !z) return 0;
  const int k = static_cast<int>(kind);
  const uint32_t total = static_cast<uint32_t>(shell_start(k, static_cast<int>(n_shells)));
  if (total > cap) return 0;
  for (uint32_t i = 0; i < total; ++i) {
    const ShellVec v = shell_vec(k, static_cast<int>(i));
    disp[3 * i + 0] = v.x;
    disp[3 * i + 1] = v.y;
    disp[3 * i + 2] = v.z;
  }
  for (uint32_t m = 0; m < n_shells; ++m) z[m] = static_cast<uint32_t>(shell_z(k, static_cast<int>(m)));
  return total;
}

void smcx_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  const U4 w = philox4x32_10(ctr[0], ctr[1], ctr[2], ctr[3], key[0], key[1]);
  out[0] = w.x;
  out[1] = w.y;
  out[2] = w.z;
  out[3] = w.w;
}

smcx_status smcx_philox_device(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint64_t key,
                               uint32_t n, uint32_t* d_out, void* cuda_stream) {
  if (!d_out && n) return fail(SMCX_EINVAL, "null output");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = launch_philox_fill(c0, c1, c2, c3, key, n, d_out, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(SMCX_ECUDA, std::string("philox fill: ") + cudaGetErrorString(e));
  return SMCX_OK;
}

}  // extern "C"
