// mm_api.cu -- host runtime and C ABI (see include/mm.h).
//
// The handle owns: a device status word, a grow-only device arena for the
// emulation workspace (digit planes, exponents, per-CTA scratch, problem
// tables, tensor maps), device buffers for the host-to-host entry point, a
// private stream for CUDA-graph capture, and a cache of instantiated graphs
// for grouped calls keyed by their full signature.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <tuple>
#include <vector>

#include "guard.cuh"
#include "launch.cuh"
#include "modular.cuh"

using mmk::Problem;

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
int round_up(int x, int a) { return (x + a - 1) / a * a; }

// The square N x N problem: every dimension and leading dimension N.
Problem square_problem(const double* A, const double* B, double* C, int N) {
  Problem p{};
  p.A = A;
  p.B = B;
  p.C = C;
  p.n = p.m = p.k = N;
  p.lda = p.ldb = p.ldc = N;
  return p;
}

// Size a problem is planned by: its largest dimension.  The accuracy of both
// emulation forms depends on the inner dimension k alone, and a plan tuned
// for size max(m, n, k) >= k is at least as accurate as one for k.
int plan_size(const Problem& p) { return std::max(p.m, std::max(p.n, p.k)); }

// ---- driver entry point for tensor-map encoding (no -lcuda link needed) ----
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2-D map over `rows` rows of `ld` bf16 elements, box = 64 x box_rows, 128-byte swizzle.
bool make_plane_map(CUtensorMap* map, const void* base, int ld, long rows, int box_rows) {
  EncodeTiledFn enc = get_encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(ld), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * 2};
  cuuint32_t box[2] = {64, static_cast<cuuint32_t>(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

struct Plan {
  int form;    // 0 native, 1 digit emulation, 2 modular emulation
  int slices;  // digit count (form 1) or moduli (form 2)
  int bn;      // emulation tile width (128 or 256)
  int groups;  // digit-pair groups per tile (0 = chosen from the SM count)
};

struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  void* table_mem = nullptr;  // device memory owned by this entry (problem tables, maps)
};

}  // namespace

struct mm_handle_s {
  int device = 0;
  int num_sms = 148;
  mm_config cfg{};
  std::string tune_path;
  std::string last_error;
  uint64_t timeout_ns = 2000000000ull;
  int* d_status = nullptr;
  // grow-only arena for the emulation workspace
  void* arena = nullptr;
  size_t arena_cap = 0;
  // host-to-host entry point buffers
  double* e2e = nullptr;
  size_t e2e_cap = 0;
  // grouped host-to-host entry point: device copies of all problems, copy
  // streams and per-chunk events
  char* ge2e = nullptr;
  size_t ge2e_cap = 0;
  cudaStream_t up_stream = nullptr, down_stream = nullptr;
  std::vector<cudaEvent_t> ge2e_events;
  // grouped calls
  cudaStream_t cap_stream = nullptr;
  std::map<std::vector<long long>, GraphEntry> graphs;
  void* grp_table = nullptr;  // non-graph grouped path: device table
  size_t grp_table_cap = 0;
  void* grp_pinned = nullptr;
  size_t grp_pinned_cap = 0;
  cudaEvent_t grp_event = nullptr;
  // grouped calls: the native problems run on a side stream, forked from and
  // joined back into the call's stream (inside the captured graph)
  cudaStream_t side_stream = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  // the accuracy certificate's launches run on their own stream, forked from
  // and joined back into the call's stream
  cudaStream_t cert_stream = nullptr;
  cudaEvent_t cert_fork = nullptr, cert_join = nullptr;
  // autotune table: N upper bound -> plan
  std::vector<std::pair<int, Plan>> tune;
  // MM_FLAG_PROFILE: events around every kernel of the last call
  bool profile = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<std::pair<int, size_t>> marks;  // (kind, index of start event; end = start + 1)
  double* probe_sink = nullptr;
};

namespace {

mm_status fail(mm_handle h, mm_status st, const std::string& msg) {
  if (h) h->last_error = msg;
  return st;
}

mm_status cuda_fail(mm_handle h, cudaError_t e, const char* what) {
  return fail(h, MM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define MM_CUDA(h, call)                                   \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #call); \
  } while (0)

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// The handle's certificate counters (64-bit, at byte 32 of its 128-byte
// status block): [0] elements recomputed natively, [1] problems recomputed whole.
unsigned long long* guard_stats(mm_handle h) { return reinterpret_cast<unsigned long long*>(h->d_status + 8); }

bool guard_on(mm_handle h) { return (h->cfg.flags & MM_FLAG_NO_GUARD) == 0; }

// ---- MM_FLAG_PROFILE --------------------------------------------------------
enum { KIND_SPLIT = 0, KIND_SLICE_GEMM = 1, KIND_NATIVE = 2, KIND_RECOMBINE = 3, KIND_CERT = 4 };
static_assert(KIND_CERT + 1 == MM_PROFILE_KINDS, "profile kinds");

void prof_reset(mm_handle h) {
  h->ev_used = 0;
  h->marks.clear();
}

// Records the start event of a kernel of `kind`; returns its mark or -1.
long prof_start(mm_handle h, cudaStream_t s, int kind) {
  if (!h->profile) return -1;
  while (h->ev_pool.size() < h->ev_used + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    h->ev_pool.push_back(e);
  }
  const size_t at = h->ev_used;
  h->ev_used += 2;
  cudaEventRecord(h->ev_pool[at], s);
  h->marks.push_back({kind, at});
  return static_cast<long>(at);
}

void prof_end(mm_handle h, cudaStream_t s, long mark) {
  if (mark >= 0) cudaEventRecord(h->ev_pool[static_cast<size_t>(mark) + 1], s);
}

// Built-in plan table (a tune file overrides it): the output of
// paper_1012_2273_gb300.autotune on a GB300 (tune/gb300.tune), which times
// every plan with the accuracy certificate on, as the mean over uniform and
// log-uniform (2^+-20) inputs -- native recomputation of what the certificate
// sends back included -- and keeps the fastest accurate one.  Below N = 256
// native FP64 is as fast; from there the modular form with 14 to 16 moduli
// (the tuner's pick per bucket; neighbouring counts are within a few percent
// of each other, 13 moduli would recompute nearly every log-uniform element
// natively).  Beyond the modular form's size limit the digit form with 6
// digits.
void default_tune(mm_handle h) {
  h->tune.clear();
  h->tune.push_back({255, Plan{0, 7, 256, 0}});
  h->tune.push_back({511, Plan{2, 15, 128, 0}});
  h->tune.push_back({767, Plan{2, 16, 128, 0}});
  h->tune.push_back({1023, Plan{2, 16, 256, 0}});
  h->tune.push_back({1535, Plan{2, 15, 256, 0}});
  h->tune.push_back({1999, Plan{2, 14, 256, 0}});
  h->tune.push_back({3071, Plan{2, 15, 256, 0}});
  h->tune.push_back({65535, Plan{2, 14, 256, 0}});
  h->tune.push_back({1 << 30, Plan{1, 6, 256, 0}});
}

// Tune file: lines "max_n form slices bn [groups]" ('#' starts a comment):
// problems with N <= max_n (first matching line) use that plan.
bool load_tune(mm_handle h, const std::string& path) {
  std::ifstream in(path);
  if (!in) return false;
  std::vector<std::pair<int, Plan>> rows;
  std::string line;
  while (std::getline(in, line)) {
    const size_t hash = line.find('#');
    if (hash != std::string::npos) line.resize(hash);
    std::istringstream ss(line);
    long maxn;
    Plan p{0, 7, 256, 0};
    if (!(ss >> maxn >> p.form >> p.slices >> p.bn)) continue;
    if (!(ss >> p.groups)) p.groups = 0;
    const int max_slices = p.form == 2 ? mmk::MOD_COUNT : 8;
    if (p.form < 0 || p.form > 3 || p.slices < (p.form == 2 ? 2 : 1) || p.slices > max_slices ||
        (p.bn != 128 && p.bn != 256) || p.groups < 0 || p.groups > 36)
      return false;
    rows.push_back({static_cast<int>(std::min<long>(maxn, 1 << 30)), p});
  }
  if (rows.empty()) return false;
  std::sort(rows.begin(), rows.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
  h->tune = rows;
  return true;
}

Plan plan_for(mm_handle h, int n) {
  Plan p = h->tune.back().second;
  for (const auto& r : h->tune)
    if (n <= r.first) {
      p = r.second;
      break;
    }
  if (h->cfg.mode == MM_NATIVE_FP64) p.form = 0;
  if (h->cfg.mode == MM_EMU_BF16 || h->cfg.mode == MM_EMU_MODULAR || h->cfg.mode == MM_EMU_INT8) {
    const int want = h->cfg.mode == MM_EMU_BF16 ? 1 : h->cfg.mode == MM_EMU_MODULAR ? 2 : 3;
    if (p.form != want) {
      // a table row of another form: keep its tile width, take this form's
      // default count
      p.slices = want == 2 ? 16 : 7;
      p.groups = 0;
    }
    p.form = want;
    if (p.bn != 128 && p.bn != 256) p.bn = 128;
  }
  if (h->cfg.slices > 0) p.slices = h->cfg.slices;
  if (p.form != 0 && n < 256) p.bn = 128;
  if (p.form == 3) p.bn = 128;  // the INT8 kernel's tiles are 128 x 128
  return p;
}

int emu_grid(mm_handle h, int total_tiles) { return std::max(1, std::min(total_tiles, h->num_sms)); }

// Largest number of digit pairs whose products can share one int32 sum.
int max_pairs_for(int n) {
  const long long per_pair = static_cast<long long>(n) * (1 << 14);  // |sum_j d d| <= n 2^14
  if (per_pair <= 0) return 64;
  const long long m = (2147483647LL) / per_pair;
  return static_cast<int>(std::min<long long>(m, 64));
}

// ---- workspace layout for a list of emulated problems -----------------------
struct Arena {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t at = off;
    off = align_up(off + bytes, kAlign);
    return at;
  }
};

mm_status ensure_arena(mm_handle h, size_t bytes) {
  if (bytes <= h->arena_cap) return MM_OK;
  // Replayed graphs point into the old arena: drop them first.
  for (auto& kv : h->graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.table_mem) cudaFree(kv.second.table_mem);
  }
  h->graphs.clear();
  if (h->arena) cudaFree(h->arena);  // implicit device synchronisation
  h->arena = nullptr;
  h->arena_cap = 0;
  // An eighth to spare for the next call's growth, when the device has it.
  size_t cap = align_up(bytes + bytes / 8, 1 << 20);
  if (cudaMalloc(&h->arena, cap) != cudaSuccess) {
    cudaGetLastError();
    cap = align_up(bytes, 1 << 20);
    if (cudaMalloc(&h->arena, cap) != cudaSuccess) {
      cudaGetLastError();
      h->arena = nullptr;
      return fail(h, MM_ERR_NOMEM, "workspace allocation of " + std::to_string(cap) + " bytes failed");
    }
  }
  h->arena_cap = cap;
  return MM_OK;
}

// Problems smaller than this recombine in a separate pass after the slice
// products (see layout_group); larger ones in the slice-product epilogue.
constexpr int kDeferBelowN = 3072;

// One launch group of the emulation: problems sharing (form, bn, groups).
struct EmuGroup {
  int form = 1;         // 1 digit form, 2 modular form
  bool tabled = false;  // launched with a device problem/unit table (grouped calls)
  int groups = 0;       // forced pair groups per tile (0 = automatic)
  int bn = 256, grid = 1, max_pairs = 1;
  bool pair = false;    // modular form at bn 256: CTA pairs (cta_group::2) on 256 x 256 tiles
  bool guard = false;   // accuracy certificate and native recomputation of what it cannot vouch for
  int guard_tiles = 0;  // blocks of the guard kernel's whole-problem part
  bool cert_folded = false;  // the certificate's products run as units of the paired kernel
  std::vector<Problem> ps;
  std::vector<int> max_off;        // offset of problem p in the maxbits arrays
  std::vector<CUtensorMap> maps;   // 2 per problem
  std::vector<int4> units;         // grouped launches: {problem, tile, group, cost}
  std::vector<int4> cert_units;    // grouped launches: the certificate's {problem, tile, 0, cost}
  int cert_total = 0;              // units of the certificate's launch
  int cert_grid = 1;               // its CTAs
  int total_tiles = 0, total_split = 0, total_absmax = 0, total_units = 0, max_rows = 0, scratch_slots = 1;
  long long tilebuf_elems = 0;
  // byte offsets inside the group's region of the arena
  size_t amax = 0, bmax = 0, scratch = 0, tilebuf = 0, counters = 0, bytes = 0;
  size_t gsum = 0;        // certificate sums and failure counts
  size_t zero_bytes = 0;  // bytes from amax on that every launch zeroes first
  char* base = nullptr;
};

// Pair groups per tile for a problem launched alone.  Estimated time =
// waves of units x the longest unit's k-blocks x the time of one k-block on
// the tensor cores, plus, when G > 1, one write and one read of every tile's
// segment slots through memory.  The constants are GB300 measurements: about
// 0.35 us per 128 x 256 x 64 k-block of digit products in steady state, and
// about 6 TB/s for streaming slot traffic.
// (The modular form writes its residue slots whatever G is, so they cost
// nothing extra there.)
int choose_groups_single(int tiles, int s, bool modular, int kb, int sms, int max_pairs) {
  const int P = modular ? mmk::mod_groups(s) : mmk::emu_pairs(s);
  const double t_kb = 0.35e-6, bw = 6.0e12, slot_bytes = 128.0 * 256.0 * 4.0;
  int best = 1;
  double best_t = 1e30;
  for (int G = 1; G <= P; ++G) {
    const long long units = static_cast<long long>(tiles) * G;
    const long long waves = (units + sms - 1) / sms;
    const int longest = (P + G - 1) / G * (modular ? 2 : 1);  // products in the longest unit
    double t = static_cast<double>(waves) * longest * kb * t_kb;
    if (G > 1 && !modular) t += 2.0 * tiles * mmk::emu_tile_slots(s, G, max_pairs) * slot_bytes / bw;
    if (t < best_t * 0.98) {  // a new group count must win by 2%
      best_t = t;
      best = G;
    }
  }
  return best;
}

// Sizes the group's workspace and work units; with `base` set, also points
// the problems into it and encodes the tensor maps.
// CTA pairs (cta_group::2) for the modular form at bn 256 only with
// The modular form at tile width 256 runs its residue products on CTA pairs
// (cta_group::2): on GB300 they measured faster than single CTAs at every
// size (the paper's sweep: 0.267 against 0.274 ms; N = 8192: 1874 against
// 1727 TFLOP/s of residue products).  MM_PAIR_MMA=0 selects the single-CTA
// kernel.
bool pair_mma_enabled() {
  const char* e = std::getenv("MM_PAIR_MMA");
  return !(e && e[0] == '0');
}

mm_status layout_group(mm_handle h, EmuGroup& g, char* base) {
  Arena ar;
  g.total_tiles = g.total_split = g.total_absmax = g.max_rows = 0;
  g.pair = g.form == 2 && g.bn == 256 && pair_mma_enabled() && h->num_sms >= 2;
  // With CTA pairs the certificate's products are units of the paired kernel
  // (one per pair tile, group index `groups`), tested in its epilogue.
  g.cert_folded = g.pair && g.guard;
  g.guard_tiles = 0;
  int maxk = 0;
  g.max_off.assign(g.ps.size(), 0);
  for (Problem& p : g.ps) maxk = std::max(maxk, p.k);
  g.max_pairs = max_pairs_for(maxk);
  long long work = 0;
  for (size_t i = 0; i < g.ps.size(); ++i) {
    Problem& p = g.ps[i];
    p.m_pad = round_up(p.m, g.pair ? 256 : 128);  // a pair covers two 128-row tiles
    p.n_pad = round_up(p.n, g.bn);
    p.k_pad = round_up(p.k, 64);
    p.tiles_m = p.m_pad / 128;
    p.tiles_n = p.n_pad / g.bn;
    p.tile_begin = g.total_tiles;
    g.total_tiles += p.tiles_m * p.tiles_n;
    p.split_begin = g.total_split;
    g.total_split += mmk::split_tiles(p);
    p.absmax_begin = g.total_absmax;
    g.total_absmax += mmk::absmax_blocks(p);
    p.beta = g.form == 2 ? mmk::mod_beta(p.s, p.k) : 0;  // the bound involves the inner dimension
    work += static_cast<long long>(p.tiles_m) * p.tiles_n * mmk::problem_pairs(p) * (p.k_pad / 64);
    // planes: s digits or residues, plus the magnitude plane when guarded
    const int planes = p.s + (g.guard ? 1 : 0);
    const size_t elt = g.form == 3 ? 1 : 2;  // int8 or bf16 digits
    p.guard = g.guard ? 1 : 0;
    p.i8 = g.form == 3 ? 1 : 0;
    const size_t a_sl = ar.take(static_cast<size_t>(planes) * p.m_pad * p.k_pad * elt);
    const size_t b_sl = ar.take(static_cast<size_t>(planes) * p.n_pad * p.k_pad * elt);
    if (g.guard) {
      // certificate constants for inner dimension k and width w (guard.cuh)
      const int w = g.form == 2 ? p.beta : g.form == 3 ? 8 * p.s - 2 : 8 * p.s - 1;
      mmk::cert_constants(p.k, w, g.form == 2 ? 0.0 : mmk::digit_kappa(p.s, w), &p.cert_k1, &p.cert_k2);
      // more failures than a quarter of the outputs: recompute the whole
      // problem natively (then the per-element list would cost about as much)
      p.guard_limit = static_cast<int>(std::min<long long>(std::max<long long>(256, static_cast<long long>(p.m) * p.n / 4),
                                                           1LL << 30));
      p.guard_tile_begin = g.guard_tiles;
      g.guard_tiles += mmk::guard_tiles(p);
    }
    const size_t ae = ar.take(sizeof(int) * p.m);
    const size_t be = ar.take(sizeof(int) * p.n);
    if (base) {
      p.a_slices = reinterpret_cast<uint16_t*>(base + a_sl);
      p.b_slices = reinterpret_cast<uint16_t*>(base + b_sl);
      p.a_exp = reinterpret_cast<int*>(base + ae);
      p.b_exp = reinterpret_cast<int*>(base + be);
    }
    g.max_off[i] = g.max_rows;  // row maxima of A (m) and column maxima of B (n) share the offset
    g.max_rows += std::max(p.m, p.n);
  }
  // Work units: pair groups per tile, then slot storage.  Grouped calls aim at
  // about MM_UNITS_PER_SM units per SM (default 4) so the dynamic scheduler
  // can balance uneven problems with a short tail.
  double units_per_sm = 4.0;
  if (const char* e = std::getenv("MM_UNITS_PER_SM")) units_per_sm = std::max(1.0, std::atof(e));
  const double target = static_cast<double>(work) / (units_per_sm * h->num_sms);
  g.units.clear();
  g.tilebuf_elems = 0;
  g.scratch_slots = 1;
  const long long slot = 128LL * g.bn;
  const bool modular = g.form == 2;
  for (size_t i = 0; i < g.ps.size(); ++i) {
    Problem& p = g.ps[i];
    const int tiles = p.tiles_m * p.tiles_n;
    // work-unit tiles: 256 x 256 pair tiles (two CTAs each) or 128-row tiles
    const int unit_tiles = g.pair ? tiles / 2 : tiles;
    const int kb = p.k_pad / 64;
    const int P = mmk::problem_pairs(p);
    int G;
    if (g.groups > 0) {
      G = std::min(g.groups, P);
    } else if (g.ps.size() == 1) {
      G = choose_groups_single(unit_tiles, p.s, modular, kb, g.pair ? h->num_sms / 2 : h->num_sms, g.max_pairs);
    } else {
      G = static_cast<int>(std::lround(P * kb / std::max(target, 1.0)));
      G = std::max(1, std::min(G, P));
    }
    if (modular) {
      // Two bytes per output and residue group (pair of moduli): ceil(k/2)
      // slots of 128 x bn 16-bit entries per tile, always recombined by the
      // separate pass.  The slots are written whatever the grouping, so
      // grouped calls give every residue group its own unit: the most,
      // equal, units for the dynamic scheduler.
      const int NG = mmk::mod_groups(p.s);
      if (g.groups == 0 && g.ps.size() > 1) G = NG;
      G = std::min(G, NG);
      p.groups = G;
      p.nslots = NG;
      p.defer = 1;
      p.slot_base = g.tilebuf_elems;
      g.tilebuf_elems += static_cast<long long>(tiles) * p.nslots * (slot / 2);
      if (g.tabled) {
        for (int gi = 0; gi < G; ++gi) {
          int p0, p1;
          mmk::mod_group_range(p.s, G, gi, &p0, &p1);
          const int cost = (p1 - p0) * kb;
          for (int t = 0; t < unit_tiles; ++t) g.units.push_back(make_int4(static_cast<int>(i), t, gi, cost));
        }
        if (g.cert_folded)
          for (int t = 0; t < unit_tiles; ++t) g.units.push_back(make_int4(static_cast<int>(i), t, G, kb));
      }
      continue;
    }
    // A tile's segment slots are listed per problem (at most 64).
    while (G > 1 && mmk::emu_tile_slots(p.s, G, g.max_pairs) > 64) --G;
    p.groups = G;
    p.nslots = mmk::emu_tile_slots(p.s, G, g.max_pairs);
    if (p.nslots > 64) return fail(h, MM_ERR_UNSUPPORTED, "too many accumulation segments for this size");
    {
      int k = 0;
      for (int gi = 0; gi < G; ++gi) {
        int p0, p1, L, t0;
        mmk::emu_group_range(p.s, G, gi, &p0, &p1);
        for (int q = p0; q < p1; ++k) {
          q += mmk::emu_segment(q, p1, g.max_pairs, &L, &t0);
          p.slot_level[k] = static_cast<int8_t>(L);
        }
      }
    }
    // Short tiles (small N) leave the recombination to a separate pass: done
    // in the epilogue it stalls the tensor pipe for a large share of the tile.
    // (the INT8 kernel always leaves the recombination to the separate pass)
    p.defer = (p.k < kDeferBelowN || g.form == 3) ? 1 : 0;  // short k loops: few k-blocks per tile
    if (G > 1 || p.defer) {
      p.slot_base = g.tilebuf_elems;
      g.tilebuf_elems += static_cast<long long>(tiles) * p.nslots * slot;
    } else {
      p.slot_base = 0;
      g.scratch_slots = std::max(g.scratch_slots, p.nslots);
    }
    if (g.tabled) {
      for (int gi = 0; gi < G; ++gi) {
        int p0, p1;
        mmk::emu_group_range(p.s, G, gi, &p0, &p1);
        const int cost = (p1 - p0) * kb;
        for (int t = 0; t < tiles; ++t) g.units.push_back(make_int4(static_cast<int>(i), t, gi, cost));
      }

    }
  }
  if (g.tabled) {
    // Longest units first, then group-major so concurrent CTAs share slices.
    std::stable_sort(g.units.begin(), g.units.end(), [](const int4& a, const int4& b) {
      if (a.w != b.w) return a.w > b.w;
      if (a.x != b.x) return a.x < b.x;
      if (a.z != b.z) return a.z < b.z;
      return a.y < b.y;
    });
    g.total_units = static_cast<int>(g.units.size());
  } else {
    g.total_units = g.ps[0].tiles_m * g.ps[0].tiles_n / (g.pair ? 2 : 1) * (g.ps[0].groups + (g.cert_folded ? 1 : 0));
  }
  g.grid = g.pair ? 2 * emu_grid(h, std::min(g.total_units, h->num_sms / 2)) : emu_grid(h, g.total_units);
  if (g.form == 3) g.grid = std::max(1, std::min(g.total_units, mmk::i8_blocks_per_sm() * h->num_sms));
  // The certificate's own launch: one unit per tile, k-blocks as the cost,
  // longest first (grouped calls list them; a single problem numbers them).
  g.cert_units.clear();
  g.cert_total = 0;
  if (g.guard && !g.cert_folded) {
    for (size_t i = 0; i < g.ps.size(); ++i) {
      const Problem& p = g.ps[i];
      const int tiles = p.tiles_m * p.tiles_n;
      if (g.tabled)
        for (int t = 0; t < tiles; ++t) g.cert_units.push_back(make_int4(static_cast<int>(i), t, 0, p.k_pad / 64));
      g.cert_total += tiles;
    }
    std::stable_sort(g.cert_units.begin(), g.cert_units.end(),
                     [](const int4& a, const int4& b) { return a.w > b.w; });
    // The two launches run side by side (the certificate on a forked
    // stream): the CTA slots are shared in proportion to their k-blocks, so
    // that both finish together instead of the certificate running in the
    // slice products' tail.  (Profiling runs them one after the other, each
    // on every slot.)
    const int slots = g.form == 3 ? mmk::i8_blocks_per_sm() * h->num_sms : h->num_sms;
    double main_kb = 0.0, cert_kb = 0.0;
    for (const Problem& p : g.ps) {
      const double kb = p.k_pad / 64.0, tiles = static_cast<double>(p.tiles_m) * p.tiles_n;
      main_kb += tiles * mmk::problem_pairs(p) * kb;
      cert_kb += tiles * kb;
    }
    g.cert_grid = std::max(1, std::min(g.cert_total, static_cast<int>(std::lround(slots * cert_kb / (main_kb + cert_kb)))));
    if (!h->profile && slots > g.cert_grid) g.grid = std::max(1, std::min(g.grid, slots - g.cert_grid));
    if (h->profile) g.cert_grid = std::min(g.cert_total, slots);
  }
  // Everything zeroed before a launch sits in one run (one memset): the
  // row/column maxima, the tile and unit counters, and -- when guarded --
  // per problem the certificate's row sums [m] and column sums [n], then the
  // per-problem failure counts and their total.
  g.amax = ar.take(sizeof(uint64_t) * g.max_rows);
  g.bmax = ar.take(sizeof(uint64_t) * g.max_rows);
  g.counters = ar.take(sizeof(int) * (8 * static_cast<size_t>(g.total_tiles) + 2));  // + unit counters (main, certificate)
  std::vector<size_t> sum_off(g.ps.size(), 0);
  size_t counts_at = 0, gsum_len = 0;
  if (g.guard) {
    for (size_t i = 0; i < g.ps.size(); ++i) {
      sum_off[i] = gsum_len;
      gsum_len += sizeof(uint64_t) * (static_cast<size_t>(g.ps[i].m) + g.ps[i].n);
    }
    counts_at = gsum_len;
    gsum_len += sizeof(int) * (g.ps.size() + 1);
  }
  g.gsum = ar.take(gsum_len);
  g.zero_bytes = ar.off - g.amax;
  g.scratch = ar.take(static_cast<size_t>(g.grid) * g.scratch_slots * slot * sizeof(int32_t));
  g.tilebuf = ar.take(static_cast<size_t>(std::max<long long>(g.tilebuf_elems, 4)) * sizeof(int32_t));
  if (g.guard) {
    for (size_t i = 0; i < g.ps.size(); ++i) {
      const size_t list_off = ar.take(sizeof(int2) * static_cast<size_t>(g.ps[i].guard_limit));
      if (!base) continue;
      Problem& p = g.ps[i];
      char* gb = base + g.gsum;
      int* counts = reinterpret_cast<int*>(gb + counts_at);
      p.a_sum = reinterpret_cast<unsigned long long*>(gb + sum_off[i]);
      p.b_sum = p.a_sum + p.m;
      p.guard_count = counts + i;
      p.guard_total = counts + g.ps.size();
      p.guard_list = reinterpret_cast<int2*>(base + list_off);
    }
  }
  g.bytes = ar.off;
  g.base = base;
  if (base) {
    // (CTA pairs stage half of a B^T tile per CTA)
    const size_t np = g.ps.size();
    g.maps.assign(2 * np, CUtensorMap{});
    for (size_t i = 0; i < np && g.form != 3; ++i) {  // (the INT8 kernel copies with cp.async)
      const Problem& p = g.ps[i];
      const long planes = p.s + (g.guard ? 1 : 0);
      if (!make_plane_map(&g.maps[2 * i], p.a_slices, p.k_pad, planes * p.m_pad, 128) ||
          !make_plane_map(&g.maps[2 * i + 1], p.b_slices, p.k_pad, planes * p.n_pad,
                          g.pair ? g.bn / 2 : g.bn))
        return fail(h, MM_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    }
  }
  return MM_OK;
}

// Enqueues the emulated path of group g: zero the maxima, scale+split, slice
// products with fused recombination.  With d_table == nullptr the group must
// hold one problem, passed by value; otherwise d_table/d_maps/d_max_off/d_units
// are device copies of g.ps, g.maps, g.max_off and g.units.
mm_status run_group(mm_handle h, const EmuGroup& g, const Problem* d_table, const CUtensorMap* d_maps,
                    const int* d_max_off, const int4* d_units, const int4* d_cert_units, cudaStream_t stream) {
  if (g.total_units == 0) return MM_OK;
  uint64_t* amax = reinterpret_cast<uint64_t*>(g.base + g.amax);
  uint64_t* bmax = reinterpret_cast<uint64_t*>(g.base + g.bmax);
  const bool single = d_table == nullptr;
  const long m_split = prof_start(h, stream, KIND_SPLIT);
  // maxima, counters and certificate sums: one run of the workspace
  MM_CUDA(h, cudaMemsetAsync(amax, 0, g.zero_bytes, stream));
  MM_CUDA(h, mmk::split_launch(d_table, single ? &g.ps[0] : nullptr, static_cast<int>(g.ps.size()), g.total_split,
                               g.total_absmax,
                               amax, bmax, single ? nullptr : d_max_off, h->d_status, stream));
  prof_end(h, stream, m_split);
  // Per-region completion counters (pair groups > 1) and the unit counter.
  int* counters = reinterpret_cast<int*>(g.base + g.counters);
  mmk::EmuArgs a{};
  a.table = d_table;
  if (single) a.single = g.ps[0];
  a.maps = d_maps;
  a.units = single ? nullptr : d_units;
  a.count = static_cast<int>(g.ps.size());
  a.total_units = g.total_units;
  a.max_pairs = g.max_pairs;
  a.scratch = reinterpret_cast<int32_t*>(g.base + g.scratch);
  a.scratch_slots = g.scratch_slots;
  a.tilebuf = reinterpret_cast<int32_t*>(g.base + g.tilebuf);
  a.tile_counters = counters;
  a.unit_counter = counters + 8 * static_cast<size_t>(g.total_tiles);
  a.levels_out = nullptr;
  a.status = h->d_status;
  a.timeout_ns = h->timeout_ns;
  // Without CTA pairs the certificate has a launch of its own, which needs
  // only the split's planes and sums.  Unless profiling, it runs on its own
  // stream beside the slice products, on the SMs they leave; the guard kernel
  // waits for it.
  bool cert_forked = false;
  if (g.guard && !g.cert_folded) {
    mmk::EmuArgs c = a;
    c.units = single ? nullptr : d_cert_units;
    c.total_units = g.cert_total;
    c.unit_counter = a.unit_counter + 1;
    cudaStream_t cs = stream;
    if (!h->profile) {
      MM_CUDA(h, cudaEventRecord(h->cert_fork, stream));
      MM_CUDA(h, cudaStreamWaitEvent(h->cert_stream, h->cert_fork, 0));
      cs = h->cert_stream;
      cert_forked = true;
    }
    const long m_c = prof_start(h, cs, KIND_CERT);
    const cudaError_t ce =
        g.form == 3 ? mmk::i8_cert_launch(c, g.cert_grid, cs)
                    : mmk::emu_cert_launch(g.bn, &g.maps[0], &g.maps[1], c, g.cert_grid, cs);
    prof_end(h, cs, m_c);
    if (ce != cudaSuccess) return cuda_fail(h, ce, "certificate launch");
    if (cert_forked) MM_CUDA(h, cudaEventRecord(h->cert_join, cs));
  }
  const long m_gemm = prof_start(h, stream, KIND_SLICE_GEMM);
  const cudaError_t le = g.form == 3 ? mmk::i8_gemm_launch(a, g.grid, stream)
                        : g.pair    ? mmk::mod_pair_gemm_launch(&g.maps[0], &g.maps[1], a, g.grid, stream)
                                    : mmk::emu_gemm_launch(g.bn, g.form == 2, &g.maps[0], &g.maps[1], a, g.grid, stream);
  prof_end(h, stream, m_gemm);
  if (le != cudaSuccess) {
    char info[512];
    mmk::emu_kernel_info(g.bn, info, sizeof(info));
    return fail(h, MM_ERR_CUDA, std::string("slice-product launch: ") + cudaGetErrorString(le) + " " + info);
  }
  if (g.form == 2) {
    // one recombination launch over the tiles of every modular problem
    const long m_rec = prof_start(h, stream, KIND_RECOMBINE);
    MM_CUDA(h, mmk::mod_recombine_launch(g.bn, a, 0, g.total_tiles, stream));
    prof_end(h, stream, m_rec);
  } else {
    bool any_deferred = false;
    for (const Problem& p : g.ps) any_deferred |= p.defer != 0;
    if (any_deferred) {
      const long m_rec = prof_start(h, stream, KIND_RECOMBINE);
      MM_CUDA(h, mmk::slots_recombine_launch(g.bn, a, g.total_tiles, stream));
      prof_end(h, stream, m_rec);
    }
  }
  if (g.guard) {
    // native FP64 for what the certificate could not vouch for (returns at
    // once when every element passed)
    if (cert_forked) MM_CUDA(h, cudaStreamWaitEvent(stream, h->cert_join, 0));
    const long m_g = prof_start(h, stream, KIND_NATIVE);
    MM_CUDA(h, mmk::guard_launch(d_table, single ? &g.ps[0] : nullptr, static_cast<int>(g.ps.size()), g.guard_tiles,
                                 h->num_sms, guard_stats(h), stream));
    prof_end(h, stream, m_g);
  }
  return MM_OK;
}

// k: the inner dimension (N of a square problem), which bounds the exact sums.
mm_status check_emu_size(mm_handle h, int k, int s, int form) {
  if (form == 2) {
    if (s < 2 || s > mmk::MOD_COUNT) return fail(h, MM_ERR_UNSUPPORTED, "the modular form takes 2..16 moduli");
    if (k > 65535) return fail(h, MM_ERR_UNSUPPORTED, "the modular form supports N (inner dimension K) <= 65535");
    if (mmk::mod_beta(s, k) < 1)
      return fail(h, MM_ERR_UNSUPPORTED, "too few moduli for this N (the fixed-point width would be 0)");
    return MM_OK;
  }
  if (s < 1 || s > 8) return fail(h, MM_ERR_UNSUPPORTED, "slices must be in 1..8");
  if (k > 131071)
    return fail(h, MM_ERR_UNSUPPORTED, "emulation supports N (inner dimension K) <= 131071 (one pair per int32 sum)");
  return MM_OK;
}

// Single emulated problem: workspace, maps, launches (no device table).
mm_status emu_single(mm_handle h, const Problem& p, int form, int s, int bn, int groups, cudaStream_t stream) {
  mm_status st = check_emu_size(h, p.k, s, form);
  if (st != MM_OK) return st;
  EmuGroup g;
  g.form = form;
  g.guard = guard_on(h);
  g.bn = bn;
  g.groups = groups;
  g.ps.push_back(p);
  g.ps[0].s = s;
  st = layout_group(h, g, nullptr);
  if (st != MM_OK) return st;
  st = ensure_arena(h, g.bytes);
  if (st != MM_OK) return st;
  st = layout_group(h, g, static_cast<char*>(h->arena));
  if (st != MM_OK) return st;
  return run_group(h, g, nullptr, nullptr, nullptr, nullptr, nullptr, stream);
}

mm_status native_single(mm_handle h, Problem p, cudaStream_t stream) {
  const bool small = mmk::native_is_small(p);
  if (small) mmk::native_small_fill_tiles(p); else mmk::native_fill_tiles(p);
  p.tile_begin = 0;
  const long m = prof_start(h, stream, KIND_NATIVE);
  if (small)
    MM_CUDA(h, mmk::native_small_launch(nullptr, &p, 1, p.tiles_m * p.tiles_n, stream,
                                        mmk::native_small_use_batch(&p, 1, h->num_sms)));
  else
    MM_CUDA(h, mmk::native_launch(nullptr, &p, 1, p.tiles_m * p.tiles_n, stream));
  prof_end(h, stream, m);
  return MM_OK;
}

// The grouped product over a list of validated problems (any shapes; m or n
// zero: skipped; k zero: C = 0).
mm_status grouped_impl(mm_handle h, const std::vector<Problem>& probs, cudaStream_t user) {
  prof_reset(h);
  const bool use_graph = (h->cfg.flags & (MM_FLAG_NO_GRAPH | MM_FLAG_PROFILE)) == 0;

  // A call identical to an earlier one replays its graph without redoing the
  // host-side planning.  (Graphs are dropped whenever the arena is regrown.)
  std::vector<long long> key;
  key.reserve(11 * probs.size() + 3);
  key.push_back(static_cast<long long>(probs.size()));
  key.push_back(h->cfg.mode);
  key.push_back(h->cfg.slices);
  for (const Problem& q : probs) {
    for (int v : {q.m, q.n, q.k, q.lda, q.ldb, q.ldc, q.ta, q.tb}) key.push_back(v);
    key.push_back(static_cast<long long>(reinterpret_cast<uintptr_t>(q.A)));
    key.push_back(static_cast<long long>(reinterpret_cast<uintptr_t>(q.B)));
    key.push_back(static_cast<long long>(reinterpret_cast<uintptr_t>(q.C)));
  }
  auto it = h->graphs.end();
  if (use_graph) {
    it = h->graphs.find(key);
    if (it != h->graphs.end()) {
      MM_CUDA(h, cudaGraphLaunch(it->second.exec, user));
      return MM_OK;
    }
  }

  // Partition: native problems, and emulated problems by (slices, bn).
  std::vector<Problem> nat;
  std::map<std::tuple<int, int, int>, std::vector<Problem>> emu;  // (form, bn, groups)
  std::vector<std::pair<Problem, Plan>> emu_plans;
  for (const Problem& q : probs) {
    if (q.m == 0 || q.n == 0) continue;
    Problem p = q;
    Plan pl = plan_for(h, plan_size(p));
    if (p.k == 0) pl.form = 0;  // C = 0: the native kernel writes it
    if (pl.form == 0) {
      nat.push_back(p);
    } else {
      mm_status st = check_emu_size(h, p.k, pl.slices, pl.form);
      if (st != MM_OK) return st;
      p.s = pl.slices;
      emu_plans.push_back({p, pl});
    }
  }
  // All emulated problems of the call share one slice-product launch: the
  // tile width is the one planned for the largest problem (digit counts may
  // differ per problem).
  if (!emu_plans.empty()) {
    size_t big = 0;
    for (size_t i = 1; i < emu_plans.size(); ++i)
      if (plan_size(emu_plans[i].first) > plan_size(emu_plans[big].first)) big = i;
    const int bn = emu_plans[big].second.bn;
    for (auto& ep : emu_plans) emu[{ep.second.form, ep.second.form == 3 ? 128 : bn, ep.second.groups}].push_back(ep.first);
  }
  // Native problems: 64 x 64 tiles, or 16 x 16 tiles below 512 (two launches).
  std::vector<Problem> nat_small;
  {
    std::vector<Problem> big;
    for (const Problem& p : nat) (mmk::native_is_small(p) ? nat_small : big).push_back(p);
    nat.swap(big);
  }
  int nat_tiles = 0, nat_small_tiles = 0;
  for (Problem& p : nat) {
    mmk::native_fill_tiles(p);
    p.tile_begin = nat_tiles;
    nat_tiles += p.tiles_m * p.tiles_n;
  }
  for (Problem& p : nat_small) {
    mmk::native_small_fill_tiles(p);
    p.tile_begin = nat_small_tiles;
    nat_small_tiles += p.tiles_m * p.tiles_n;
  }

  // Workspace.  Emulation groups run one after another on the same stream, so
  // they all start at offset 0 of the arena; a group whose workspace exceeds
  // the limit is cut into waves (largest problems first), each run in turn.
  size_t limit = 0;
  {
    size_t free_b = 0, total_b = 0;
    if (const char* e = std::getenv("MM_WORKSPACE_LIMIT_MB")) limit = static_cast<size_t>(std::atoll(e)) << 20;
    if (!limit && cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
      const size_t reserve = size_t(1) << 30;
      limit = h->arena_cap + (free_b > reserve ? (free_b - reserve) / 10 * 9 : 0);
    }
    cudaGetLastError();
    if (!limit) limit = size_t(64) << 30;
  }
  std::vector<EmuGroup> groups;
  size_t arena_need = 0;
  for (auto& kv : emu) {
    std::vector<Problem> rest = kv.second;
    std::stable_sort(rest.begin(), rest.end(), [](const Problem& a, const Problem& b) {
      return static_cast<double>(a.m) * a.n * a.k > static_cast<double>(b.m) * b.n * b.k;
    });
    size_t at = 0;
    while (at < rest.size()) {
      // Largest prefix of the remaining problems whose workspace fits the
      // limit (binary search; at least one problem).
      auto make = [&](size_t end) {
        EmuGroup t;
        t.tabled = true;
        t.guard = guard_on(h);
        t.form = std::get<0>(kv.first);
        t.bn = std::get<1>(kv.first);
        t.groups = std::get<2>(kv.first);
        t.ps.assign(rest.begin() + at, rest.begin() + end);
        return t;
      };
      EmuGroup g = make(rest.size());
      mm_status st = layout_group(h, g, nullptr);
      if (st != MM_OK) return st;
      size_t end = rest.size();
      if (g.bytes > limit && rest.size() - at > 1) {
        size_t lo = at + 1, hi = rest.size() - 1;  // lo always fits or is the single-problem floor
        while (lo < hi) {
          const size_t mid = (lo + hi + 1) / 2;
          EmuGroup t = make(mid);
          st = layout_group(h, t, nullptr);
          if (st != MM_OK) return st;
          if (t.bytes <= limit) lo = mid; else hi = mid - 1;
        }
        end = lo;
        g = make(end);
        st = layout_group(h, g, nullptr);
        if (st != MM_OK) return st;
      }
      at = end;
      arena_need = std::max(arena_need, g.bytes);
      groups.push_back(std::move(g));
    }
  }
  if (arena_need) {
    mm_status st = ensure_arena(h, arena_need);
    if (st != MM_OK) return st;
  }
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    mm_status st = layout_group(h, groups[gi], static_cast<char*>(h->arena));
    if (st != MM_OK) return st;
  }

  // Device-side tables: [native problems][per group: problems, maps, max offsets].
  Arena tab;
  const size_t off_nat = tab.take(sizeof(Problem) * std::max<size_t>(nat.size(), 1));
  const size_t off_nat_small = tab.take(sizeof(Problem) * std::max<size_t>(nat_small.size(), 1));
  std::vector<size_t> off_tab, off_maps, off_mo, off_units, off_cert;
  for (const EmuGroup& g : groups) {
    off_tab.push_back(tab.take(sizeof(Problem) * g.ps.size()));
    off_maps.push_back(tab.take(sizeof(CUtensorMap) * g.maps.size()));
    off_mo.push_back(tab.take(sizeof(int) * g.max_off.size()));
    off_units.push_back(tab.take(sizeof(int4) * std::max<size_t>(g.units.size(), 1)));
    off_cert.push_back(tab.take(sizeof(int4) * std::max<size_t>(g.cert_units.size(), 1)));
  }
  const size_t tab_bytes = tab.off;
  std::vector<char> host_tab(tab_bytes, 0);
  if (!nat.empty()) std::memcpy(host_tab.data() + off_nat, nat.data(), sizeof(Problem) * nat.size());
  if (!nat_small.empty())
    std::memcpy(host_tab.data() + off_nat_small, nat_small.data(), sizeof(Problem) * nat_small.size());
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    const EmuGroup& g = groups[gi];
    std::memcpy(host_tab.data() + off_tab[gi], g.ps.data(), sizeof(Problem) * g.ps.size());
    std::memcpy(host_tab.data() + off_maps[gi], g.maps.data(), sizeof(CUtensorMap) * g.maps.size());
    std::memcpy(host_tab.data() + off_mo[gi], g.max_off.data(), sizeof(int) * g.max_off.size());
    if (!g.units.empty()) std::memcpy(host_tab.data() + off_units[gi], g.units.data(), sizeof(int4) * g.units.size());
    if (!g.cert_units.empty())
      std::memcpy(host_tab.data() + off_cert[gi], g.cert_units.data(), sizeof(int4) * g.cert_units.size());
  }

  const bool nat_batch =
      !nat_small.empty() && mmk::native_small_use_batch(nat_small.data(), static_cast<int>(nat_small.size()), h->num_sms);
  auto launch_all = [&](char* dtab, cudaStream_t s) -> mm_status {
    // Native problems do not depend on the emulation's kernels: unless
    // profiling (which wants one kernel at a time), they run on a side stream.
    const bool fork = !h->profile && (!nat.empty() || !nat_small.empty()) && !groups.empty();
    if (fork) {
      MM_CUDA(h, cudaEventRecord(h->fork_ev, s));
      MM_CUDA(h, cudaStreamWaitEvent(h->side_stream, h->fork_ev, 0));
      if (!nat_small.empty())
        MM_CUDA(h, mmk::native_small_launch(reinterpret_cast<Problem*>(dtab + off_nat_small), nullptr,
                                            static_cast<int>(nat_small.size()), nat_small_tiles, h->side_stream,
                                            nat_batch));
      if (!nat.empty())
        MM_CUDA(h, mmk::native_launch(reinterpret_cast<Problem*>(dtab + off_nat), nullptr,
                                      static_cast<int>(nat.size()), nat_tiles, h->side_stream));
      MM_CUDA(h, cudaEventRecord(h->join_ev, h->side_stream));
    } else if (!nat.empty() || !nat_small.empty()) {
      const long m = prof_start(h, s, KIND_NATIVE);
      if (!nat_small.empty())
        MM_CUDA(h, mmk::native_small_launch(reinterpret_cast<Problem*>(dtab + off_nat_small), nullptr,
                                            static_cast<int>(nat_small.size()), nat_small_tiles, s, nat_batch));
      if (!nat.empty())
        MM_CUDA(h, mmk::native_launch(reinterpret_cast<Problem*>(dtab + off_nat), nullptr,
                                      static_cast<int>(nat.size()), nat_tiles, s));
      prof_end(h, s, m);
    }
    for (size_t gi = 0; gi < groups.size(); ++gi) {
      mm_status st = run_group(h, groups[gi], reinterpret_cast<Problem*>(dtab + off_tab[gi]),
                               reinterpret_cast<CUtensorMap*>(dtab + off_maps[gi]),
                               reinterpret_cast<int*>(dtab + off_mo[gi]),
                               reinterpret_cast<int4*>(dtab + off_units[gi]),
                               reinterpret_cast<int4*>(dtab + off_cert[gi]), s);
      if (st != MM_OK) return st;
    }
    if (fork) MM_CUDA(h, cudaStreamWaitEvent(s, h->join_ev, 0));
    return MM_OK;
  };

  if (!use_graph) {
    if (tab_bytes > h->grp_table_cap) {
      if (h->grp_table) cudaFree(h->grp_table);
      if (h->grp_pinned) cudaFreeHost(h->grp_pinned);
      h->grp_table = nullptr;
      h->grp_pinned = nullptr;
      h->grp_table_cap = 0;
      if (cudaMalloc(&h->grp_table, tab_bytes) != cudaSuccess ||
          cudaMallocHost(&h->grp_pinned, tab_bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, MM_ERR_NOMEM, "grouped table buffers");
      }
      h->grp_table_cap = tab_bytes;
    }
    MM_CUDA(h, cudaEventSynchronize(h->grp_event));  // previous upload done with the staging buffer
    std::memcpy(h->grp_pinned, host_tab.data(), tab_bytes);
    MM_CUDA(h, cudaMemcpyAsync(h->grp_table, h->grp_pinned, tab_bytes, cudaMemcpyHostToDevice, user));
    MM_CUDA(h, cudaEventRecord(h->grp_event, user));
    return launch_all(static_cast<char*>(h->grp_table), user);
  }

  it = h->graphs.find(key);  // the arena may have been regrown above (cache cleared)
  if (it == h->graphs.end()) {
    if (h->graphs.size() >= 32) {
      for (auto& kv : h->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.table_mem) cudaFree(kv.second.table_mem);
      }
      h->graphs.clear();
    }
    GraphEntry ge;
    if (cudaMalloc(&ge.table_mem, std::max<size_t>(tab_bytes, 256)) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, MM_ERR_NOMEM, "grouped table");
    }
    if (cudaMemcpy(ge.table_mem, host_tab.data(), tab_bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaFree(ge.table_mem);
      return fail(h, MM_ERR_CUDA, "grouped table upload");
    }
    cudaGraph_t graph = nullptr;
    MM_CUDA(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    mm_status st = launch_all(static_cast<char*>(ge.table_mem), h->cap_stream);
    cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &graph);
    if (st != MM_OK || ce != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaFree(ge.table_mem);
      cudaGetLastError();
      return st != MM_OK ? st : cuda_fail(h, ce, "graph capture");
    }
    ce = cudaGraphInstantiate(&ge.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
      cudaFree(ge.table_mem);
      return cuda_fail(h, ce, "graph instantiate");
    }
    it = h->graphs.emplace(key, ge).first;
  }
  MM_CUDA(h, cudaGraphLaunch(it->second.exec, user));
  return MM_OK;
}

// Validates one problem of the _ex entry points and fills *p.  op(A) is
// m x k and op(B) k x n; ta / tb: A / B is stored as the transpose (k x m,
// n x k).  m or n zero (or k zero with a valid C) is accepted; pointers need
// only be 8-byte aligned (no kernel reads A, B or C with wider accesses).
mm_status make_rect_problem(mm_handle h, int ta, int tb, int m, int n, int k, const double* A, int lda, const double* B,
                            int ldb, double* C, int ldc, Problem* p) {
  if (m < 0 || n < 0 || k < 0) return fail(h, MM_ERR_INVALID, "M, N, K must be >= 0");
  if ((ta != 0 && ta != 1) || (tb != 0 && tb != 1)) return fail(h, MM_ERR_INVALID, "transa, transb must be 0 or 1");
  *p = Problem{};
  p->m = m;
  p->n = n;
  p->k = k;
  if (m == 0 || n == 0) return MM_OK;
  if (!C || (k > 0 && (!A || !B))) return fail(h, MM_ERR_INVALID, "null matrix pointer");
  // stored shapes (rows x columns)
  const int a_rows = ta ? k : m, a_cols = ta ? m : k;
  const int b_rows = tb ? n : k, b_cols = tb ? k : n;
  if (ldc < n || (k > 0 && (lda < a_cols || ldb < b_cols)))
    return fail(h, MM_ERR_INVALID, "leading dimensions must be at least the stored row lengths");
  auto al8 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 7u) == 0; };
  if (!al8(C) || (k > 0 && (!al8(A) || !al8(B)))) return fail(h, MM_ERR_INVALID, "pointers must be 8-byte aligned");
  // C's span must not meet A's or B's
  auto span = [](const void* base, int rows, int cols, int ld) {
    const char* b = static_cast<const char*>(base);
    return std::make_pair(b, b + (static_cast<size_t>(rows - 1) * ld + cols) * sizeof(double));
  };
  const auto c = span(C, m, n, ldc);
  if (k > 0) {
    const auto a = span(A, a_rows, a_cols, lda), b = span(B, b_rows, b_cols, ldb);
    if ((c.first < a.second && a.first < c.second) || (c.first < b.second && b.first < c.second))
      return fail(h, MM_ERR_INVALID, "C must not overlap A or B");
  }
  p->A = A;
  p->B = B;
  p->C = C;
  p->lda = k > 0 ? lda : 1;
  p->ldb = k > 0 ? ldb : 1;
  p->ldc = ldc;
  p->ta = ta;
  p->tb = tb;
  return MM_OK;
}

// One problem, alone: the native or emulated path of its plan.
mm_status single_impl(mm_handle h, const Problem& p, cudaStream_t s) {
  if (p.m == 0 || p.n == 0) return MM_OK;
  prof_reset(h);
  Plan plan = plan_for(h, plan_size(p));
  if (p.k == 0) plan.form = 0;  // C = 0: the native kernel writes it
  if (plan.form == 0) return native_single(h, p, s);
  return emu_single(h, p, plan.form, plan.slices, plan.bn, plan.groups, s);
}

}  // namespace

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

mm_status mm_create(mm_handle* out, const mm_config* cfg) {
  if (!out) return MM_ERR_INVALID;
  *out = nullptr;
  mm_handle h = new (std::nothrow) mm_handle_s();
  if (!h) return MM_ERR_NOMEM;
  h->cfg.mode = MM_AUTO;
  h->cfg.slices = 0;
  h->cfg.flags = 0;
  h->cfg.tune_path = nullptr;
  if (cfg) {
    h->cfg = *cfg;
    if (cfg->tune_path) h->tune_path = cfg->tune_path;
    h->cfg.tune_path = nullptr;
  }
  if (h->cfg.mode != MM_NATIVE_FP64 && h->cfg.mode != MM_EMU_BF16 && h->cfg.mode != MM_AUTO &&
      h->cfg.mode != MM_EMU_MODULAR && h->cfg.mode != MM_EMU_INT8) {
    delete h;
    return MM_ERR_INVALID;
  }
  if (h->cfg.slices < 0 || h->cfg.slices > (h->cfg.mode == MM_EMU_MODULAR ? mmk::MOD_COUNT : 8) ||
      (h->cfg.mode == MM_EMU_MODULAR && h->cfg.slices == 1)) {
    delete h;
    return MM_ERR_UNSUPPORTED;
  }
  if (const char* t = std::getenv("MM_TIMEOUT_MS")) {  // milliseconds, fractions allowed
    const double ms = std::atof(t);
    if (ms > 0) h->timeout_ns = std::max<uint64_t>(100, static_cast<uint64_t>(ms * 1e6));
  }
  h->profile = (h->cfg.flags & MM_FLAG_PROFILE) != 0;
  default_tune(h);
  if (!h->tune_path.empty() && !load_tune(h, h->tune_path)) {
    delete h;
    return MM_ERR_INVALID;
  }
  if (cudaGetDevice(&h->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess ||
      cudaMalloc(&h->d_status, 128) != cudaSuccess || cudaMemset(h->d_status, 0, 128) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->cert_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->cert_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->cert_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->join_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->grp_event, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (h->d_status) cudaFree(h->d_status);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    delete h;
    return MM_ERR_CUDA;
  }
  *out = h;
  return MM_OK;
}

mm_status mm_destroy(mm_handle h) {
  if (!h) return MM_ERR_INVALID;
  cudaDeviceSynchronize();
  for (auto& kv : h->graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.table_mem) cudaFree(kv.second.table_mem);
  }
  if (h->arena) cudaFree(h->arena);
  if (h->e2e) cudaFree(h->e2e);
  if (h->ge2e) cudaFree(h->ge2e);
  if (h->up_stream) cudaStreamDestroy(h->up_stream);
  if (h->down_stream) cudaStreamDestroy(h->down_stream);
  for (cudaEvent_t e : h->ge2e_events) cudaEventDestroy(e);
  if (h->grp_table) cudaFree(h->grp_table);
  if (h->grp_pinned) cudaFreeHost(h->grp_pinned);
  if (h->grp_event) cudaEventDestroy(h->grp_event);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->side_stream) cudaStreamDestroy(h->side_stream);
  if (h->cert_stream) cudaStreamDestroy(h->cert_stream);
  if (h->cert_fork) cudaEventDestroy(h->cert_fork);
  if (h->cert_join) cudaEventDestroy(h->cert_join);
  if (h->fork_ev) cudaEventDestroy(h->fork_ev);
  if (h->join_ev) cudaEventDestroy(h->join_ev);
  if (h->d_status) cudaFree(h->d_status);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  if (h->probe_sink) cudaFree(h->probe_sink);
  delete h;
  return MM_OK;
}

mm_status mm_profile_read(mm_handle h, double out_ms[MM_PROFILE_KINDS], int launches[MM_PROFILE_KINDS]) {
  if (!h || !out_ms) return MM_ERR_INVALID;
  if (!h->profile) return fail(h, MM_ERR_INVALID, "handle was created without MM_FLAG_PROFILE");
  for (int k = 0; k < MM_PROFILE_KINDS; ++k) {
    out_ms[k] = 0.0;
    if (launches) launches[k] = 0;
  }
  for (const auto& m : h->marks) {
    cudaEvent_t e0 = h->ev_pool[m.second], e1 = h->ev_pool[m.second + 1];
    MM_CUDA(h, cudaEventSynchronize(e1));
    float ms = 0.f;
    MM_CUDA(h, cudaEventElapsedTime(&ms, e0, e1));
    out_ms[m.first] += ms;
    if (launches) launches[m.first] += (m.first == KIND_SPLIT) ? 2 : 1;  // split = absmax + split kernels
  }
  return MM_OK;
}

mm_status mm_selftest_wait(mm_handle h, int timeout_ms, void* stream) {
  if (!h || timeout_ms <= 0 || timeout_ms > 60000) return MM_ERR_INVALID;
  MM_CUDA(h, mmk::selftest_wait(h->d_status, static_cast<uint64_t>(timeout_ms) * 1000000ull, nullptr,
                                static_cast<cudaStream_t>(stream)));
  return MM_OK;
}

mm_status mm_probe_fp64_peak(mm_handle h, double* dmma_tflops, double* dfma_tflops) {
  if (!h || !dmma_tflops || !dfma_tflops) return MM_ERR_INVALID;
  if (!h->probe_sink) MM_CUDA(h, cudaMalloc(&h->probe_sink, 64));
  MM_CUDA(h, mmk::probe_fp64(h->num_sms, h->probe_sink, h->cap_stream, dmma_tflops, dfma_tflops));
  return MM_OK;
}

mm_status mm_probe_int8_peak(mm_handle h, double* tops) {
  if (!h || !tops) return MM_ERR_INVALID;
  if (!h->probe_sink) MM_CUDA(h, cudaMalloc(&h->probe_sink, 64));
  MM_CUDA(h, mmk::probe_int8(h->num_sms, reinterpret_cast<int*>(h->probe_sink), h->cap_stream, tops));
  return MM_OK;
}

const char* mm_last_error(mm_handle h) { return h ? h->last_error.c_str() : "invalid handle"; }

mm_status mm_modular_params(int k, int N, int* beta, int* moduli) {
  if (k < 1 || k > mmk::MOD_COUNT || N < 1 || !beta) return MM_ERR_INVALID;
  *beta = mmk::mod_beta(k, N);
  if (moduli)
    for (int j = 0; j < k; ++j) moduli[j] = static_cast<int>(mmk::mod_value(j));
  return MM_OK;
}

mm_status mm_plan(mm_handle h, int N, int* form, int* slices) {
  if (!h || N < 0) return MM_ERR_INVALID;
  const Plan p = plan_for(h, N);
  if (form) *form = p.form;
  if (slices) *slices = p.slices;
  return MM_OK;
}

mm_status mm_status_get(mm_handle h, void* stream) {
  if (!h) return MM_ERR_INVALID;
  MM_CUDA(h, cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  int st = 0;
  MM_CUDA(h, cudaMemcpy(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st != 0) {
    MM_CUDA(h, cudaMemset(h->d_status, 0, sizeof(int)));
    return fail(h, static_cast<mm_status>(st), st == MM_ERR_TIMEOUT ? "a device-side wait timed out"
                                             : st == MM_ERR_NONFINITE ? "non-finite input to the emulation"
                                                                      : "device error");
  }
  return MM_OK;
}

mm_status mm_guard_read(mm_handle h, void* stream, long long* elements, long long* problems) {
  if (!h) return MM_ERR_INVALID;
  MM_CUDA(h, cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  unsigned long long v[2] = {0, 0};
  MM_CUDA(h, cudaMemcpy(v, guard_stats(h), sizeof(v), cudaMemcpyDeviceToHost));
  MM_CUDA(h, cudaMemset(guard_stats(h), 0, sizeof(v)));
  if (elements) *elements = static_cast<long long>(v[0]);
  if (problems) *problems = static_cast<long long>(v[1]);
  return MM_OK;
}

mm_status mm_gemm(mm_handle h, int N, const double* A, const double* B, double* C, void* stream) {
  if (!h) return MM_ERR_INVALID;
  if (N < 0) return fail(h, MM_ERR_INVALID, "N must be >= 0");
  if (N == 0) return MM_OK;
  if (!A || !B || !C) return fail(h, MM_ERR_INVALID, "null matrix pointer");
  if (!aligned16(A) || !aligned16(B) || !aligned16(C)) return fail(h, MM_ERR_INVALID, "pointers must be 16-byte aligned");
  const size_t bytes = static_cast<size_t>(N) * N * sizeof(double);
  auto overlap = [bytes](const void* x, const void* y) {
    const char* a = static_cast<const char*>(x);
    const char* b = static_cast<const char*>(y);
    return a < b + bytes && b < a + bytes;
  };
  if (overlap(C, A) || overlap(C, B)) return fail(h, MM_ERR_INVALID, "C must not overlap A or B");
  return single_impl(h, square_problem(A, B, C, N), static_cast<cudaStream_t>(stream));
}

mm_status mm_gemm_ex(mm_handle h, int transa, int transb, int M, int N, int K, const double* A, int lda,
                     const double* B, int ldb, double* C, int ldc, void* stream) {
  if (!h) return MM_ERR_INVALID;
  Problem p{};
  const mm_status st = make_rect_problem(h, transa, transb, M, N, K, A, lda, B, ldb, C, ldc, &p);
  if (st != MM_OK) return st;
  return single_impl(h, p, static_cast<cudaStream_t>(stream));
}

mm_status mm_gemm_host(mm_handle h, int N, const double* A_host, const double* B_host, double* C_host,
                       void* stream) {
  if (!h) return MM_ERR_INVALID;
  if (N < 0 || (N > 0 && (!A_host || !B_host || !C_host))) return fail(h, MM_ERR_INVALID, "bad arguments");
  if (N == 0) return MM_OK;
  const size_t elems = static_cast<size_t>(N) * N;
  const size_t need = 3 * align_up(elems * sizeof(double), kAlign);
  if (need > h->e2e_cap) {
    if (h->e2e) cudaFree(h->e2e);
    h->e2e = nullptr;
    h->e2e_cap = 0;
    if (cudaMalloc(&h->e2e, need) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, MM_ERR_NOMEM, "device buffers for the host entry point");
    }
    h->e2e_cap = need;
  }
  const size_t stride = align_up(elems * sizeof(double), kAlign) / sizeof(double);
  double* dA = h->e2e;
  double* dB = h->e2e + stride;
  double* dC = h->e2e + 2 * stride;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // Once a copy is enqueued it may still be reading or writing the caller's
  // host buffers: every way out from here waits for the stream first.
  auto drain = [&](mm_status st) {
    cudaStreamSynchronize(s);
    cudaGetLastError();
    return st;
  };
  cudaError_t e = cudaMemcpyAsync(dA, A_host, elems * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dB, B_host, elems * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return drain(cuda_fail(h, e, "upload of A or B"));
  const mm_status st = mm_gemm(h, N, dA, dB, dC, stream);
  if (st != MM_OK) return drain(st);
  e = cudaMemcpyAsync(C_host, dC, elems * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return drain(cuda_fail(h, e, "download of C"));
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return drain(cuda_fail(h, e, "cudaStreamSynchronize"));
  return MM_OK;
}

mm_status mm_gemm_grouped_host(mm_handle h, int count, const int* Ns, const double* const* As_host,
                               const double* const* Bs_host, double* const* Cs_host, void* stream) {
  if (!h) return MM_ERR_INVALID;
  if (count < 0) return fail(h, MM_ERR_INVALID, "count must be >= 0");
  if (count == 0) return MM_OK;
  if (!Ns || !As_host || !Bs_host || !Cs_host) return fail(h, MM_ERR_INVALID, "null array");
  for (int i = 0; i < count; ++i) {
    if (Ns[i] < 0) return fail(h, MM_ERR_INVALID, "negative N in group");
    if (Ns[i] > 0 && (!As_host[i] || !Bs_host[i] || !Cs_host[i])) return fail(h, MM_ERR_INVALID, "null matrix in group");
  }
  // Device copies: A, B, C of every problem, 256-byte aligned.
  std::vector<size_t> off(count, 0);
  size_t need = 0;
  for (int i = 0; i < count; ++i) {
    off[i] = need;
    need += 3 * align_up(static_cast<size_t>(Ns[i]) * Ns[i] * sizeof(double), kAlign);
  }
  if (need > h->ge2e_cap) {
    if (h->ge2e) cudaFree(h->ge2e);
    h->ge2e = nullptr;
    h->ge2e_cap = 0;
    if (cudaMalloc(&h->ge2e, need) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, MM_ERR_NOMEM, "device buffers for the grouped host entry point");
    }
    h->ge2e_cap = need;
  }
  if (!h->up_stream) {
    if (cudaStreamCreateWithFlags(&h->up_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->down_stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, MM_ERR_CUDA, "copy streams");
    }
  }
  // Chunks, in decreasing problem size: the products take longer than the
  // copies, so the largest computation starts first and the uploads of the
  // rest overlap it, and the last chunk -- whose product and download
  // nothing overlaps -- holds the smallest problems.  Leading chunks close
  // once they hold a quarter of the work (at most three of them); the
  // remaining problems form the last chunk.  (On GB300 the paper's sweep as
  // [2000], [1500], [the rest] took 1.025 ms end to end, against 1.116 ms
  // with the small problems first.)
  std::vector<int> order;
  double total = 0.0;
  for (int i = 0; i < count; ++i) {
    if (Ns[i] <= 0) continue;
    order.push_back(i);
    total += 2.0 * Ns[i] * static_cast<double>(Ns[i]) * Ns[i];
  }
  if (order.empty()) return MM_OK;
  std::stable_sort(order.begin(), order.end(), [Ns](int a, int b) { return Ns[a] > Ns[b]; });
  std::vector<std::vector<int>> chunks(1);
  double in_chunk = 0.0;
  for (int i : order) {
    if (chunks.size() <= 3 && in_chunk >= total / 4.0) {
      chunks.emplace_back();
      in_chunk = 0.0;
    }
    chunks.back().push_back(i);
    in_chunk += 2.0 * Ns[i] * static_cast<double>(Ns[i]) * Ns[i];
  }
  while (h->ge2e_events.size() < 2 * chunks.size() + 1) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, MM_ERR_CUDA, "events");
    }
    h->ge2e_events.push_back(e);
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t start = h->ge2e_events[2 * chunks.size()];
  MM_CUDA(h, cudaEventRecord(start, s));  // earlier work on the caller's stream comes first
  MM_CUDA(h, cudaStreamWaitEvent(h->up_stream, start, 0));
  // From here on, copies that touch the caller's host buffers may be in
  // flight: every way out waits for them first.
  auto drain = [&](mm_status st) {
    cudaStreamSynchronize(h->up_stream);
    cudaStreamSynchronize(h->down_stream);
    cudaStreamSynchronize(s);
    cudaGetLastError();
    return st;
  };
#define MM_CUDA_DRAIN(call)                                              \
  do {                                                                   \
    cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess) return drain(cuda_fail(h, e_, #call));        \
  } while (0)
  auto dptr = [&](int i, int which) {
    const size_t bytes = align_up(static_cast<size_t>(Ns[i]) * Ns[i] * sizeof(double), kAlign);
    return reinterpret_cast<double*>(h->ge2e + off[i] + which * bytes);
  };
  for (size_t c = 0; c < chunks.size(); ++c) {
    cudaEvent_t in = h->ge2e_events[2 * c], done = h->ge2e_events[2 * c + 1];
    std::vector<int> cn;
    std::vector<const double*> ca, cb;
    std::vector<double*> cc;
    for (int i : chunks[c]) {
      const size_t bytes = static_cast<size_t>(Ns[i]) * Ns[i] * sizeof(double);
      MM_CUDA_DRAIN(cudaMemcpyAsync(dptr(i, 0), As_host[i], bytes, cudaMemcpyHostToDevice, h->up_stream));
      MM_CUDA_DRAIN(cudaMemcpyAsync(dptr(i, 1), Bs_host[i], bytes, cudaMemcpyHostToDevice, h->up_stream));
      cn.push_back(Ns[i]);
      ca.push_back(dptr(i, 0));
      cb.push_back(dptr(i, 1));
      cc.push_back(dptr(i, 2));
    }
    MM_CUDA_DRAIN(cudaEventRecord(in, h->up_stream));
    MM_CUDA_DRAIN(cudaStreamWaitEvent(s, in, 0));
    const mm_status st = mm_gemm_grouped(h, static_cast<int>(cn.size()), cn.data(), ca.data(), cb.data(), cc.data(), s);
    if (st != MM_OK) return drain(st);
    MM_CUDA_DRAIN(cudaEventRecord(done, s));
    MM_CUDA_DRAIN(cudaStreamWaitEvent(h->down_stream, done, 0));
    for (size_t q = 0; q < chunks[c].size(); ++q) {
      const int i = chunks[c][q];
      MM_CUDA_DRAIN(cudaMemcpyAsync(Cs_host[i], cc[q], static_cast<size_t>(Ns[i]) * Ns[i] * sizeof(double),
                                 cudaMemcpyDeviceToHost, h->down_stream));
    }
  }
  MM_CUDA_DRAIN(cudaStreamSynchronize(h->down_stream));
  MM_CUDA_DRAIN(cudaStreamSynchronize(s));
#undef MM_CUDA_DRAIN
  return MM_OK;
}

mm_status mm_gemm_grouped(mm_handle h, int count, const int* Ns, const double* const* As, const double* const* Bs,
                          double* const* Cs, void* stream) {
  if (!h) return MM_ERR_INVALID;
  if (count < 0) return fail(h, MM_ERR_INVALID, "count must be >= 0");
  if (count == 0) return MM_OK;
  if (!Ns || !As || !Bs || !Cs) return fail(h, MM_ERR_INVALID, "null array");
  std::vector<Problem> probs;
  probs.reserve(count);
  for (int i = 0; i < count; ++i) {
    if (Ns[i] < 0) return fail(h, MM_ERR_INVALID, "negative N in group");
    if (Ns[i] > 0 && (!As[i] || !Bs[i] || !Cs[i])) return fail(h, MM_ERR_INVALID, "null matrix in group");
    if (Ns[i] > 0 && (!aligned16(As[i]) || !aligned16(Bs[i]) || !aligned16(Cs[i])))
      return fail(h, MM_ERR_INVALID, "group pointers must be 16-byte aligned");
    probs.push_back(square_problem(As[i], Bs[i], Cs[i], Ns[i]));
  }
  return grouped_impl(h, probs, static_cast<cudaStream_t>(stream));
}

mm_status mm_gemm_grouped_ex(mm_handle h, int count, const int* transas, const int* transbs, const int* Ms,
                             const int* Ns, const int* Ks, const double* const* As, const int* ldas,
                             const double* const* Bs, const int* ldbs, double* const* Cs, const int* ldcs,
                             void* stream) {
  if (!h) return MM_ERR_INVALID;
  if (count < 0) return fail(h, MM_ERR_INVALID, "count must be >= 0");
  if (count == 0) return MM_OK;
  if (!Ms || !Ns || !Ks || !As || !ldas || !Bs || !ldbs || !Cs || !ldcs) return fail(h, MM_ERR_INVALID, "null array");
  std::vector<Problem> probs;
  probs.reserve(count);
  for (int i = 0; i < count; ++i) {
    Problem p{};
    mm_status st = make_rect_problem(h, transas ? transas[i] : 0, transbs ? transbs[i] : 0, Ms[i], Ns[i], Ks[i], As[i],
                                     ldas[i], Bs[i], ldbs[i], Cs[i], ldcs[i], &p);
    if (st != MM_OK) return st;
    probs.push_back(p);
  }
  return grouped_impl(h, probs, static_cast<cudaStream_t>(stream));
}

mm_status mm_split(mm_handle h, int N, const double* M, int by_columns, int slices, int* exps, uint16_t* digits,
                   int rows, int ld, void* stream) {
  if (!h) return MM_ERR_INVALID;
  if (N <= 0 || !M || !exps || !digits || rows < N || ld < N || rows % 128 || ld % 64 || !aligned16(digits))
    return fail(h, MM_ERR_INVALID, "mm_split: bad arguments (rows % 128, ld % 64, 16-byte aligned digits)");
  if (slices < 1 || slices > 8) return fail(h, MM_ERR_UNSUPPORTED, "slices must be in 1..8");
  Problem p = square_problem(nullptr, nullptr, nullptr, N);
  p.s = slices;
  p.k_pad = ld;
  if (by_columns) {
    p.B = M;
    p.b_slices = digits;
    p.b_exp = exps;
    p.n_pad = rows;
    p.m_pad = 0;
  } else {
    p.A = M;
    p.a_slices = digits;
    p.a_exp = exps;
    p.m_pad = rows;
    p.n_pad = 0;
  }
  const size_t need = 2 * align_up(sizeof(uint64_t) * N, kAlign);
  mm_status st = ensure_arena(h, need);
  if (st != MM_OK) return st;
  uint64_t* mx = static_cast<uint64_t*>(h->arena);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  MM_CUDA(h, cudaMemsetAsync(mx, 0, sizeof(uint64_t) * N, s));
  MM_CUDA(h, mmk::split_launch(nullptr, &p, 1, mmk::split_tiles(p), 0, mx, mx, nullptr, h->d_status, s));
  return MM_OK;
}

mm_status mm_level_sums(mm_handle h, int N, int slices, const uint16_t* a_digits, int a_rows,
                        const uint16_t* b_digits, int b_rows, int ld, int32_t* levels, void* stream) {
  if (!h) return MM_ERR_INVALID;
  if (N <= 0 || !a_digits || !b_digits || !levels || a_rows < N || b_rows < N || ld < N || a_rows % 128 ||
      b_rows % 128 || ld % 64)
    return fail(h, MM_ERR_INVALID, "mm_level_sums: bad arguments");
  if (slices < 1 || slices > 8) return fail(h, MM_ERR_UNSUPPORTED, "slices must be in 1..8");
  if (static_cast<long long>(slices) * N * (1 << 14) >= (1LL << 31))
    return fail(h, MM_ERR_UNSUPPORTED, "level sums would not fit int32");
  const int bn = (b_rows % 256 == 0 && N > 128) ? 256 : 128;
  Problem p = square_problem(nullptr, nullptr, nullptr, N);
  p.s = slices;
  p.a_slices = const_cast<uint16_t*>(a_digits);
  p.b_slices = const_cast<uint16_t*>(b_digits);
  p.m_pad = a_rows;
  p.n_pad = b_rows;
  p.k_pad = ld;
  p.tiles_m = (N + 127) / 128;
  p.tiles_n = (N + bn - 1) / bn;
  p.tile_begin = 0;
  p.groups = 1;
  p.nslots = slices;
  std::vector<CUtensorMap> maps(2);
  if (!make_plane_map(&maps[0], a_digits, ld, static_cast<long>(slices) * a_rows, 128) ||
      !make_plane_map(&maps[1], b_digits, ld, static_cast<long>(slices) * b_rows, bn))
    return fail(h, MM_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  mmk::EmuArgs a{};
  a.single = p;
  a.count = 1;
  a.total_units = p.tiles_m * p.tiles_n;
  a.max_pairs = slices;  // every level in one segment: level sums fit int32 (checked above)
  a.scratch = nullptr;
  a.scratch_slots = 0;
  a.unit_counter = h->d_status + 16;  // spare word of the status block
  MM_CUDA(h, cudaMemsetAsync(a.unit_counter, 0, sizeof(int), static_cast<cudaStream_t>(stream)));
  a.levels_out = levels;
  a.status = h->d_status;
  a.timeout_ns = h->timeout_ns;
  const cudaError_t le = mmk::emu_gemm_launch(bn, false, &maps[0], &maps[1], a, emu_grid(h, a.total_units),
                                              static_cast<cudaStream_t>(stream));
  if (le != cudaSuccess) {
    char info[512];
    mmk::emu_kernel_info(bn, info, sizeof(info));
    return fail(h, MM_ERR_CUDA, std::string("slice-product launch: ") + cudaGetErrorString(le) + " " + info);
  }
  return MM_OK;
}

mm_status mm_recombine(mm_handle h, int N, int slices, const int32_t* levels, const int* a_exps, const int* b_exps,
                       double* C, void* stream) {
  if (!h) return MM_ERR_INVALID;
  if (N <= 0 || !levels || !a_exps || !b_exps || !C) return fail(h, MM_ERR_INVALID, "mm_recombine: bad arguments");
  if (slices < 1 || slices > 8) return fail(h, MM_ERR_UNSUPPORTED, "slices must be in 1..8");
  prof_reset(h);
  const long m = prof_start(h, static_cast<cudaStream_t>(stream), KIND_RECOMBINE);
  MM_CUDA(h, mmk::recombine_launch(N, slices, levels, a_exps, b_exps, C, static_cast<cudaStream_t>(stream)));
  prof_end(h, static_cast<cudaStream_t>(stream), m);
  return MM_OK;
}

}  // extern "C"
