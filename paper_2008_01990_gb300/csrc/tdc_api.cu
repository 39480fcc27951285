// tdc_api.cu -- the C ABI (include/tdc.h): argument checks, the host plan of
// the divide-and-conquer tree, the workspace layout and the launch sequence.
//
// The tree of a problem of order n has depth t (the smallest t with
// ceil(n/2^t) <= leaf) and node boundaries floor(i n / 2^l) on level l
// (Algorithm 1's recursive split, written level by level).  Every kernel of a
// merge level processes all nodes of that level of all problems at once; each
// level's roots side runs on the caller's stream and its products side on a
// second stream, so that the roots of one level overlap the products of the
// level below (run_plan).
#include <algorithm>
#include <array>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "tdc_common.cuh"

namespace tdc {

// Device-side status.  Every stream that calls the library gets a slot of two words
// in a fixed device array (assigned on its first call; loaded with the library, so no
// allocation): the first error and the warning bits.  A call clears its stream's slot
// when it is enqueued and its kernels write there, so tdc_sync_status(stream) reads
// the status of the last call on that stream and of no other, whatever became of the
// call's workspace.  With more streams than slots, later streams share the last slot.
constexpr int kStatusSlots = 1024;
__device__ int g_status_slots[kStatusSlots][2];

static std::mutex g_mu;
static int* g_slots_base[64];                            // device address of the slot array per device
static int g_slots_used[64];
static int* g_last_slot[64];                             // slot of the last call per device
static std::map<std::pair<int, cudaStream_t>, int*> g_stream_slot;  // slot of each stream
static tdc_stats g_last_stats;

// The slot of (current device, stream), assigned on first use; NULL on failure.
static int* stream_slot(cudaStream_t s, bool assign) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_slots_base[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_status_slots) != cudaSuccess || !p) return nullptr;
    g_slots_base[dev] = (int*)p;
  }
  auto it = g_stream_slot.find({dev, s});
  if (it != g_stream_slot.end()) return it->second;
  if (!assign) return g_last_slot[dev];
  const int idx = std::min(g_slots_used[dev], kStatusSlots - 1);
  if (g_slots_used[dev] < kStatusSlots) ++g_slots_used[dev];
  int* slot = g_slots_base[dev] + 2 * idx;
  g_stream_slot[{dev, s}] = slot;
  return slot;
}

// Calls made inside a composed call (tdc_syevd) keep the status the outer call cleared.
static thread_local int g_status_nest = 0;
struct StatusNest {
  StatusNest() { ++g_status_nest; }
  ~StatusNest() { --g_status_nest; }
};

// Clear the stream's status slot (stream-ordered) and note it as the device's last.
static int* begin_status(cudaStream_t s) {
  int* slot = stream_slot(s, true);
  if (!slot) return nullptr;
  if (g_status_nest == 0 && cudaMemsetAsync(slot, 0, 2 * sizeof(int), s) != cudaSuccess) return nullptr;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_mu);
  g_last_slot[dev] = slot;
  return slot;
}

static int depth_of(int64_t n, int leaf) {
  int t = 0;
  while (((n + (((int64_t)1) << t) - 1) >> t) > leaf) ++t;
  return t;
}

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

// ---------------------------------------------------------------------------
// Host plan
// ---------------------------------------------------------------------------
struct HostPlan {
  std::vector<Problem> prob;  // sorted by depth, deepest first
  int64_t N = 0;              // vector slots
  int64_t Q1 = 0;             // doubles of the internal Q buffer
  int64_t nleaves = 0;
  int max_leaf = 1;
  int T = 0;                  // levels
  std::vector<LevelLaunch> levels;  // index l
  int64_t Mmax = 1;
  std::vector<int64_t> max_tiles;   // GEMM tile upper bound per level
  int64_t img_elems = 0;            // digit images of the split path (bf16 elements)
  int64_t max_passes = 0;           // most split passes of a level
  int split_S = 0;                  // 0: split path off
  std::vector<std::vector<std::pair<int64_t, int64_t>>> split_chunks;  // per level: merge ranges
  int struct_m = 0;                 // 0: structured path off
  int64_t struct_slots = 0;         // SRRSC slots (segments x Tmax^2)
  int64_t struct_w = 0;             // W doubles
  int64_t struct_segs = 0;          // segments
  // structured path on the split GEMM (TDC_MERGE_STRUCTURED_SPLIT): largest level
  bool ss = false;
  int64_t ss_items = 0;             // segments x Tmax
  int64_t ss_bcap = 0;              // W columns (and W-product columns)
  int64_t ss_w = 0;                 // W doubles
  int64_t ss_r = 0;                 // R doubles
  int64_t ss_img = 0;               // digit-image elements of the largest of the three products
  std::vector<char> ss_level;       // per level: its structured merges take that path
  std::vector<int64_t> ss_wcap;     // per level: W columns it may use
};

// the structured path on the split GEMM: W columns per tile of a level, on average
// (tiles beyond the budget stay dense), and the digit-image elements a level may use
static constexpr int64_t kSsRankBudget = 8;
static constexpr int64_t kSsImgBudget = (int64_t)8 << 30;

// Digit-image elements of the structured path on the split GEMM for nseg parts of at
// most `rows` rows and kmax poles, `items` column tiles in all, tiles of m: one A
// image per part (read by its near and W products), with the larger of the near and
// W products' B images after it; then the apply products' own images, which reuse
// the buffer.  A near range holds at most 3m poles, a row tile at most m, and the W
// and apply products at most wcap columns / rows in all.
static int64_t ss_img_bound(int64_t nseg, int64_t items, int64_t rows, int64_t kmax, int64_t m, int64_t wcap,
                            int64_t S) {
  const int64_t at = (int64_t)kSplitBM * kSplitBK, bt = (int64_t)kSplitBN * kSplitBK;
  const int64_t RT = (rows + kSplitBM - 1) / kSplitBM, CTm = (m + kSplitBN - 1) / kSplitBN;
  const int64_t imgA = nseg * RT * ((kmax + kSplitBK - 1) / kSplitBK) * S * at;
  const int64_t nearB = items * CTm * ((3 * m + kSplitBK - 1) / kSplitBK + 2) * S * bt;
  const int64_t wB = (wcap / kSplitBN + items) * ((m + kSplitBK - 1) / kSplitBK + 2) * S * bt;
  const int64_t ap = (wcap / kSplitBK + items) * (RT * at + CTm * bt) * S;
  return std::max(imgA + std::max(nearB, wB), ap);
}

// AUTO takes the structured path on the split GEMM for merges with K >= structured_min_K
static bool struct_split_mode(const tdc_opts& o) {
  return o.merge_mode == TDC_MERGE_STRUCTURED_SPLIT || o.merge_mode == TDC_MERGE_AUTO;
}
static bool struct_enabled(const tdc_opts& o) {
  return o.merge_mode == TDC_MERGE_STRUCTURED || struct_split_mode(o);
}
// merges with K >= this take the structured path (on the split GEMM it never starts
// below the split threshold)
static int struct_threshold(const tdc_opts& o) {
  return struct_split_mode(o) ? std::max(o.structured_min_K, o.split_min_K) : o.structured_min_K;
}

static void level_struct_dims(const LevelLaunch& L, int m, int64_t& Tmax, int64_t& ldw) {
  Tmax = (L.max_n + m - 1) / m;
  ldw = (L.max_n + 1) / 2;
}

static void plan_struct(HostPlan& H, const tdc_opts& o) {
  H.struct_m = struct_enabled(o) ? o.lr_tile : 0;
  H.struct_slots = H.struct_w = H.struct_segs = 0;
  H.ss = struct_split_mode(o);
  H.ss_items = H.ss_bcap = H.ss_w = H.ss_r = H.ss_img = 0;
  H.ss_level.assign(H.T, 0);
  H.ss_wcap.assign(H.T, 0);
  if (!H.struct_m) return;
  const int64_t m = H.struct_m, S = o.split_slices;
  for (int l = 0; l < H.T; ++l) {
    const LevelLaunch& L = H.levels[l];
    if (L.max_n < struct_threshold(o)) continue;
    int64_t Tmax, ldw;
    level_struct_dims(L, H.struct_m, Tmax, ldw);
    const int64_t nseg = 2 * L.merges;
    H.struct_slots = std::max(H.struct_slots, nseg * Tmax * Tmax);
    if (!H.ss) H.struct_w = std::max(H.struct_w, nseg * Tmax * kStructRmax * ldw);
    H.struct_segs = std::max(H.struct_segs, nseg + 1);
    if (!H.ss) continue;
    // W budget: on average kSsRankBudget columns per tile of the level, at most 4 GiB
    // (tiles beyond it stay dense, in FP64); the R blocks, column lists and digit
    // images follow from it.  A row tile holds at most m poles, the near range of a
    // column tile at most 3m.
    const int64_t items = nseg * Tmax;
    const int64_t wcap = std::max<int64_t>(
        kSplitBN, std::min<int64_t>(items * Tmax * kSsRankBudget, ((int64_t)1 << 29) / std::max<int64_t>(ldw, 1)));
    const int64_t img = ss_img_bound(nseg, items, ldw, L.max_n, m, wcap, S);
    H.ss_level[l] = img <= kSsImgBudget;
    if (!H.ss_level[l]) continue;  // this level's merges take the split path
    H.ss_wcap[l] = wcap;
    H.ss_items = std::max(H.ss_items, items);
    H.ss_bcap = std::max(H.ss_bcap, wcap);
    H.ss_w = std::max(H.ss_w, wcap * ldw);
    H.ss_r = std::max(H.ss_r, wcap * m);
    H.ss_img = std::max(H.ss_img, img);
  }
  H.img_elems = std::max(H.img_elems, H.ss_img);
}

// the split path is used for merge_mode SPLIT and AUTO
static bool split_enabled(const tdc_opts& o) {
  return o.merge_mode == TDC_MERGE_SPLIT || o.merge_mode == TDC_MERGE_AUTO ||
         o.merge_mode == TDC_MERGE_STRUCTURED_SPLIT;
}

// Digit images of a merge of order nm on the split path (upper bound: kk, K <= nm).
static int64_t merge_img_bound(int64_t nm, int S) {
  const int64_t n1 = (nm + 1) / 2;
  return split_img_elems(n1, n1, nm, nm, S);
}

// The split path materialises digit images for the merges of a level; many-problem
// levels are processed in chunks of consecutive merges whose images fit a cap
// (at least the largest single merge).
static constexpr int64_t kSplitImgCap = (int64_t)4 << 30;  // bf16 elements (8 GiB)

static void plan_split(HostPlan& H, const tdc_opts& o) {
  H.img_elems = 0;
  H.max_passes = 0;
  H.split_S = split_enabled(o) ? o.split_slices : 0;
  H.split_chunks.assign(H.T, {});
  if (!H.split_S) return;
  int64_t biggest = 0;
  for (int l = 0; l < H.T; ++l)
    for (auto& p : H.prob) {
      if (p.depth <= l) break;
      const int64_t nm = (p.n + (((int64_t)1) << l) - 1) >> l;
      if (nm >= o.split_min_K) biggest = std::max(biggest, merge_img_bound(nm, H.split_S));
    }
  const int64_t cap = std::max(kSplitImgCap, biggest);
  for (int l = 0; l < H.T; ++l) {
    const LevelLaunch& L = H.levels[l];
    if (L.max_n < o.split_min_K) continue;
    int64_t g = 0, start = 0, acc = 0;
    for (int pi = 0; pi < L.nprob_act; ++pi) {
      const Problem& p = H.prob[pi];
      const int64_t nm = (p.n + (((int64_t)1) << l) - 1) >> l;
      const int64_t per = nm >= o.split_min_K ? merge_img_bound(nm, H.split_S) : 0;
      for (int64_t i = 0; i < (((int64_t)1) << l); ++i, ++g) {
        if (acc + per > cap && g > start) {
          H.split_chunks[l].push_back({start, g});
          H.img_elems = std::max(H.img_elems, acc);
          start = g;
          acc = 0;
        }
        acc += per;
      }
    }
    if (g > start) {
      H.split_chunks[l].push_back({start, g});
      H.img_elems = std::max(H.img_elems, acc);
    }
    H.max_passes = std::max(H.max_passes, (int64_t)H.split_chunks[l].size());
  }
}

static void build_plan(HostPlan& H, int32_t batch, const int64_t* n_host, const int64_t* off_de,
                       const int64_t* off_q, const int64_t* ld0, int leaf) {
  std::vector<Problem> v;
  for (int32_t b = 0; b < batch; ++b) {
    if (n_host[b] <= 0) continue;
    Problem p;
    memset(&p, 0, sizeof(p));
    p.n = n_host[b];
    p.off_de = off_de ? off_de[b] : 0;
    p.off_q = off_q ? off_q[b] : 0;
    p.ld0 = ld0 ? ld0[b] : p.n;
    p.depth = depth_of(p.n, leaf);
    v.push_back(p);
  }
  std::stable_sort(v.begin(), v.end(), [](const Problem& a, const Problem& b) { return a.depth > b.depth; });
  int64_t vo = 0, qo = 0, lf = 0;
  int T = 0, ml = 1;
  for (auto& p : v) {
    p.voff = vo;
    p.qoff1 = qo;
    p.leaf0 = lf;
    vo += p.n;
    qo += p.n * p.n;
    lf += ((int64_t)1) << p.depth;
    T = std::max(T, (int)p.depth);
    ml = std::max(ml, (int)((p.n + (((int64_t)1) << p.depth) - 1) >> p.depth));
  }
  H.prob = v;
  H.N = vo;
  H.Q1 = qo;
  H.nleaves = lf;
  H.max_leaf = ml;
  H.T = T;
  H.levels.assign(T, LevelLaunch{});
  H.max_tiles.assign(T, 0);
  H.Mmax = 1;
  for (int l = 0; l < T; ++l) {
    LevelLaunch& L = H.levels[l];
    L.level = l;
    int32_t c = 0;
    int64_t slots = 0, mx = 0, mn = INT64_MAX, tiles = 0;
    for (auto& p : v) {
      if (p.depth <= l) break;
      ++c;
      slots += p.n;
      const int64_t nm = (p.n + (((int64_t)1) << l) - 1) >> l;
      mx = std::max(mx, nm);
      mn = std::min(mn, p.n >> l);
      const int64_t n1 = (nm + 1) / 2;
      int bm, bn;
      dense_tile_dims(nm, bm, bn);
      const int64_t rt = 2 * ((n1 + bm - 1) / bm);
      tiles += (((int64_t)1) << l) * rt * ((nm + bn - 1) / bn);
    }
    L.nprob_act = c;
    L.merges = ((int64_t)c) << l;
    L.nslots = slots;
    L.max_n = mx;
    L.min_n = c > 0 ? mn : 0;
    H.max_tiles[l] = tiles;
    H.Mmax = std::max(H.Mmax, L.merges);
  }
}

// workspace carving
struct Layout {
  size_t prob, vec_d, vec_i, vec_b, minfo, tiles, stats, segs, img, srank, spiv, sy, svr, scolpiv, sw;
  size_t ss_segs, ss_counts, ss_wcol0, ss_bcol, ss_wpos, ss_w, ss_r, ss_cexp, ss_item, ss_accept, q1, total;
};

static constexpr int kVecD = 27;  // doubles per slot (13 vectors, 2 for rcs, 2 for skey, xlo, zz, 8 boundary rows)
static constexpr int kVecI = 16;  // int32 per slot (incl. 4 for rij, 2 for stag)
static constexpr int kVecB = 3;   // bytes per slot

// int64 words of one set of merge prefixes: tiles, roots, root blocks, image offsets, split passes
static int64_t tiles_per_set(const HostPlan& H) { return 4 * H.Mmax + 5 + 2 * H.max_passes + 2; }

static Layout layout_of(const HostPlan& H) {
  Layout L;
  size_t o = 0;
  L.prob = o; o = align_up(o + sizeof(Problem) * std::max<size_t>(1, H.prob.size()));
  // two sets of the per-level vectors and merge data, by level parity: a level reads
  // its children's results from the other set
  L.vec_d = o; o = align_up(o + 2 * sizeof(double) * kVecD * (size_t)std::max<int64_t>(1, H.N));
  L.vec_i = o; o = align_up(o + 2 * sizeof(int32_t) * kVecI * (size_t)std::max<int64_t>(1, H.N));
  L.vec_b = o; o = align_up(o + 2 * kVecB * (size_t)std::max<int64_t>(1, H.N));
  L.minfo = o; o = align_up(o + 2 * sizeof(int32_t) * 6 * (size_t)std::max<int64_t>(1, H.Mmax));
  L.tiles = o; o = align_up(o + 2 * sizeof(int64_t) * tiles_per_set(H));
  L.stats = o; o = align_up(o + sizeof(Stats));
  L.segs = o; o = align_up(o + ((H.split_S || H.struct_m) ? sizeof(GemmSeg) * (size_t)(2 * H.Mmax + 1) : 0));
  L.img = o; o = align_up(o + sizeof(__nv_bfloat16) * (size_t)H.img_elems);
  const size_t ns = (size_t)H.struct_slots, mm = (size_t)H.struct_m;
  L.srank = o; o = align_up(o + sizeof(int) * ns);
  L.spiv = o; o = align_up(o + sizeof(int) * ns * kStructRmax);
  L.sy = o; o = align_up(o + sizeof(double) * ns * kStructRmax);
  L.svr = o; o = align_up(o + sizeof(double) * ns * mm);
  L.scolpiv = o; o = align_up(o + sizeof(int) * ns * mm);
  L.sw = o; o = align_up(o + sizeof(double) * (size_t)H.struct_w);
  const size_t it = (size_t)H.ss_items;
  L.ss_segs = o; o = align_up(o + (H.ss ? 4 * sizeof(GemmSeg) * (it + 1) : 0));
  L.ss_counts = o; o = align_up(o + (H.ss ? 4 * sizeof(int64_t) : 0));
  L.ss_wcol0 = o; o = align_up(o + sizeof(int32_t) * ns);
  L.ss_bcol = o; o = align_up(o + sizeof(int32_t) * (size_t)H.ss_bcap);
  L.ss_wpos = o; o = align_up(o + sizeof(int32_t) * (size_t)H.ss_bcap);
  L.ss_w = o; o = align_up(o + sizeof(double) * (size_t)H.ss_w);
  L.ss_r = o; o = align_up(o + sizeof(double) * (size_t)H.ss_r);
  L.ss_cexp = o; o = align_up(o + sizeof(int32_t) * it * mm);
  L.ss_item = o; o = align_up(o + sizeof(int64_t) * 6 * it);
  L.ss_accept = o; o = align_up(o + (H.ss ? sizeof(int32_t) * 2 * (size_t)H.Mmax : 0));
  L.q1 = o; o = align_up(o + sizeof(double) * (size_t)H.Q1);
  L.total = o + 256;  // slack for aligning an unaligned base
  return L;
}

// Set k (0 or 1) of the per-level vectors and merge data.
static void carve_set(Vecs& v, MergeInfo& m, const HostPlan& H, const Layout& L, char* base, int k) {
  const size_t N = (size_t)std::max<int64_t>(1, H.N);
  double* vd = (double*)(base + L.vec_d) + (size_t)k * kVecD * N;
  v.dmod = vd + 0 * N; v.lam = vd + 1 * N; v.Dc = vd + 2 * N; v.zc = vd + 3 * N;
  v.Ds = vd + 4 * N; v.zs = vd + 5 * N; v.Dk = vd + 6 * N; v.zk = vd + 7 * N;
  v.tau = vd + 8 * N; v.zhat = vd + 9 * N; v.scol = vd + 10 * N; v.xz = (float2*)(vd + 11 * N);
  v.dval = vd + 12 * N; v.rcs = vd + 13 * N;  // rcs: 2 per slot (13N..15N)
  v.skey = vd + 15 * N;                        // 2 per slot (15N..17N)
  v.xlo = (float*)(vd + 17 * N);
  v.zz = vd + 18 * N;
  v.bf = vd + 19 * N; v.bl = vd + 20 * N; v.rbf = vd + 21 * N; v.rbl = vd + 22 * N;
  v.pf = vd + 23 * N; v.pl = vd + 24 * N; v.rf = vd + 25 * N; v.rl = vd + 26 * N;
  int32_t* vi = (int32_t*)(base + L.vec_i) + (size_t)k * kVecI * N;
  v.perm = vi + 0 * N; v.kept = vi + 1 * N; v.org = vi + 2 * N; v.dcol = vi + 3 * N;
  v.tlist = vi + 4 * N; v.blist = vi + 5 * N; v.posr = vi + 6 * N; v.posd = vi + 7 * N;
  v.rch = vi + 8 * N; v.stag = vi + 9 * N;  // 2N
  v.rij = vi + 11 * N;                       // 4N (ends at 15N)
  uint8_t* vb = (uint8_t*)(base + L.vec_b) + (size_t)k * kVecB * N;
  v.kseg = vb; v.dseg = vb + N; v.cseg = vb + 2 * N;
  const size_t M = (size_t)std::max<int64_t>(1, H.Mmax);
  int32_t* mi = (int32_t*)(base + L.minfo) + (size_t)k * 6 * M;
  m.K = mi; m.nd = mi + M; m.nrot = mi + 2 * M; m.ntop = mi + 3 * M; m.nbot = mi + 4 * M;
  m.nchain = mi + 5 * M;
  m.tiles = (int64_t*)(base + L.tiles) + (size_t)k * tiles_per_set(H);
  m.roff = m.tiles + (H.Mmax + 1);
  m.boff = m.roff + (H.Mmax + 2);
  m.ioff = m.boff + (H.Mmax + 1);
  m.spass = m.ioff + (H.Mmax + 1);
  m.sseg = m.spass + (2 * H.max_passes + 1);
}

static void carve(Plan& P, const HostPlan& H, const Layout& L, char* base) {
  Vecs v1;
  MergeInfo m1;
  carve_set(P.v, P.m, H, L, base, 0);
  carve_set(v1, m1, H, L, base, 1);
  P.lam2[0] = P.v.lam; P.lam2[1] = v1.lam;
  P.bf2[0] = P.v.bf; P.bf2[1] = v1.bf;
  P.bl2[0] = P.v.bl; P.bl2[1] = v1.bl;
  P.clam = v1.lam; P.cbf = v1.bf; P.cbl = v1.bl;
  P.Q1 = (double*)(base + L.q1);
  P.prob = (const Problem*)(base + L.prob);
  P.segs = (H.split_S || H.struct_m) ? (GemmSeg*)(base + L.segs) : nullptr;
  P.img = (__nv_bfloat16*)(base + L.img);
  P.img_cap = H.img_elems;
}

// Problem table upload through kernel parameters (capture-safe: the values
// are copied into the launch).  440 entries of 64 bytes fill most of the 32 KB of
// parameters a launch may carry, so a 4096-problem batch takes 10 launches.
static constexpr int kProbChunk = 440;
static_assert(sizeof(Problem) == 64, "problem table entry");
struct ProbChunk {
  Problem p[kProbChunk];
};
__global__ void __launch_bounds__(512) k_write_problems(ProbChunk c, int cnt, Problem* dst) {
  if (threadIdx.x < cnt) dst[threadIdx.x] = c.p[threadIdx.x];
}

static cudaError_t upload_problems(const HostPlan& H, Problem* dst, cudaStream_t s) {
  const int n = (int)H.prob.size();
  for (int b = 0; b < n; b += kProbChunk) {
    ProbChunk c;
    const int cnt = std::min(kProbChunk, n - b);
    memset(&c, 0, sizeof(c));
    for (int i = 0; i < cnt; ++i) c.p[i] = H.prob[b + i];
    k_write_problems<<<1, 512, 0, s>>>(c, cnt, dst + b);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static int validate_opts(const tdc_opts* o) {
  if (o->leaf < 2 || o->leaf > 64) return 1;  // leaf >= 2 keeps every tree node non-empty
  if (o->merge_mode < 0 || o->merge_mode > 4) return 1;
  if (o->max_iter < 1) return 1;
  if (o->lr_tile < 64 || o->lr_tile > 4096 || (o->lr_tile % 64) != 0) return 1;
  if (o->split_slices < 3 || o->split_slices > 7) return 1;
  if (o->split_min_K < 1) return 1;
  if (o->split_chunk_k < 0 || (o->split_chunk_k % 16) != 0) return 1;
  if (o->spin_budget < 1) return 1;
  if (!(o->lr_tol > 0.0)) return 1;
  return 0;
}

// Events ordering the two streams level by level: a pool per host thread and device,
// created on first use and reused by every later call (a re-recorded event stands for
// its latest record, and a call's waits are enqueued after its own records).
static cudaError_t level_events(int T, cudaEvent_t** evE, cudaEvent_t** evG, cudaEvent_t** evR) {
  static thread_local std::vector<cudaEvent_t> pool[16];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 16) return cudaErrorInvalidDevice;
  std::vector<cudaEvent_t>& v = pool[dev];
  while ((int)v.size() < 3 * T) {
    cudaEvent_t ev = nullptr;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    v.push_back(ev);
  }
  *evE = v.data();
  *evG = v.data() + T;
  *evR = v.data() + 2 * T;
  return cudaSuccess;
}

// The second stream of the solver, one per host thread and device, created on first
// use with the highest priority (the products are the critical path).
static cudaStream_t gemm_stream() {
  static thread_local cudaStream_t st[16] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 16) return nullptr;
  if (st[dev] == nullptr) {
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (cudaStreamCreateWithPriority(&st[dev], cudaStreamNonBlocking, hi) != cudaSuccess) st[dev] = nullptr;
  }
  return st[dev];
}

static int run_plan(HostPlan& H, const tdc_opts& o, const double* d, const double* e, double* lam, double* Q,
                    void* ws, size_t ws_bytes, cudaStream_t s) {
  Layout L = layout_of(H);
  if (ws == nullptr || ws_bytes < L.total) return TDC_ENOWS;
  char* base = (char*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
  Plan P;
  memset(&P, 0, sizeof(P));
  carve(P, H, L, base);
  P.nprob = (int32_t)H.prob.size();
  P.leaf = o.leaf;
  P.nslots = H.N;
  P.Q0 = Q;
  P.d = d;
  P.e = e;
  P.lam_out = lam;
  P.max_iter = o.max_iter;
  P.split_min_K = H.split_S ? o.split_min_K : 0;
  P.split_slices = H.split_S ? H.split_S : 7;
  P.split_chunk_steps = o.split_chunk_k / 16;
  P.spin_budget = o.spin_budget;
  P.struct_min_K = H.struct_m ? struct_threshold(o) : 0;
  P.struct_m = H.struct_m;
  P.struct_split = 0;  // set per level below
  StructArgs SA;
  memset(&SA, 0, sizeof(SA));
  SA.m = H.struct_m;
  SA.rmax = kStructRmax;
  SA.tol = o.lr_tol;
  SA.srank = (int*)(base + L.srank);
  SA.spiv = (int*)(base + L.spiv);
  SA.sy = (double*)(base + L.sy);
  SA.svr = (double*)(base + L.svr);
  SA.scolpiv = (int*)(base + L.scolpiv);
  SA.W = (double*)(base + L.sw);
  P.stats = o.collect_stats ? (Stats*)(base + L.stats) : nullptr;
  if (H.N == 0) return TDC_OK;
  P.status = begin_status(s);
  if (!P.status) return TDC_ECUDA;
  // PP[k]: the plan of the levels of parity k (their vectors in set k, the children's
  // in the other); PP[0] also serves the leaves and the output
  Plan PP[2] = {P, P};
  carve_set(PP[1].v, PP[1].m, H, L, base, 1);
  PP[1].clam = P.v.lam;
  PP[1].cbf = P.v.bf;
  PP[1].cbl = P.v.bl;
  cudaError_t err = upload_problems(H, (Problem*)P.prob, s);
  if (err == cudaSuccess && P.stats) err = cudaMemsetAsync(P.stats, 0, sizeof(Stats), s);
  // Phase timing (statistics only): events recorded on the call's stream.
  const bool timing = o.collect_stats != 0;
  std::vector<cudaEvent_t> evs;
  std::vector<std::pair<int, std::pair<size_t, size_t>>> spans;  // (phase, (from, to))
  auto mark_on = [&](cudaStream_t st) -> size_t {
    if (!timing) return 0;
    cudaEvent_t ev;
    cudaEventCreate(&ev);
    cudaEventRecord(ev, st);
    evs.push_back(ev);
    return evs.size() - 1;
  };
  auto mark = [&]() -> size_t { return mark_on(s); };
  auto span = [&](int phase, size_t a0, size_t a1) {
    if (timing) spans.push_back({phase, {a0, a1}});
  };
  // kernel launches: problem upload, input scale, corner modification, leaves, 9 per level (14
  // on levels that also run the thread-per-root variants), output
  int64_t launches = (int64_t)((H.prob.size() + kProbChunk - 1) / kProbChunk) + 4 + 9 * (int64_t)H.T;
  for (int l = 0; l < H.T; ++l) {
    if (l > 0) launches += 2;  // boundary rows: rotation and gather, output order
    if (H.levels[l].nslots >= kSmallMinSlots) launches += 5;
    if (H.levels[l].merges > 0 && H.levels[l].min_n <= kTinyN) launches += 1;
    if (H.split_S && H.levels[l].max_n >= o.split_min_K)
      launches += 4 * (int64_t)H.split_chunks[l].size() + (H.split_chunks[l].size() > 1 ? 1 : 0);
    if (H.struct_m && H.levels[l].max_n >= o.structured_min_K)
      launches += 2 + 2 * ((H.levels[l].max_n + H.struct_m - 1) / H.struct_m);
  }
  const size_t t0 = mark();
  if (err == cudaSuccess) err = launch_dmod(P, s);
  if (err == cudaSuccess) err = launch_leaves(P, H.nleaves, H.max_leaf, s);
  span(0, t0, mark());
  // Two streams.  The caller's stream s runs each level's roots and vectors
  // (deflation, secular equation, zhat, normalisers, ordering, boundary rows); a
  // second stream sg runs its products and copies (rotations of the children's
  // columns, FP64 / split / structured products, deflated copies).  The roots of
  // level l-1 need only level l's boundary rows, so they run on s while level l's
  // products run on sg.  Level l's products wait for its roots (evE); level l-2's
  // roots reuse level l's vector set and wait for its products (evG); the output
  // waits for the top level's products.  The rotations of the children's columns need
  // only the deflation's lists, so they wait for the deflation alone (evR) and run while
  // the level's secular equation is solved.
  cudaStream_t sg = gemm_stream();
  if (sg == nullptr) err = cudaErrorUnknown;
  cudaEvent_t* evE = nullptr;
  cudaEvent_t* evG = nullptr;
  cudaEvent_t* evR = nullptr;
  if (err == cudaSuccess) err = level_events(H.T, &evE, &evG, &evR);
  for (int l = H.T - 1; l >= 0 && err == cudaSuccess; --l) {
    const LevelLaunch& LL = H.levels[l];
    Plan P = PP[l & 1];
    const bool ss = H.ss && H.ss_level[l] && LL.max_n >= P.struct_min_K;
    P.struct_split = ss ? 1 : 0;
    if (l + 2 < H.T) err = cudaStreamWaitEvent(s, evG[l + 2], 0);
    const size_t a0 = mark();
    if (err == cudaSuccess) err = launch_prepare(P, LL, s);
    if (err == cudaSuccess) err = launch_boundary_rot(P, LL, s);
    if (err == cudaSuccess) err = cudaEventRecord(evR[l], s);
    const size_t a1 = mark();
    if (err == cudaSuccess) err = launch_secular(P, LL, s);
    const size_t a2 = mark();
    if (err == cudaSuccess) err = launch_lowner(P, LL, s);
    if (err == cudaSuccess) err = launch_finalize(P, LL, s);
    if (err == cudaSuccess) err = launch_boundary_out(P, LL, s);
    const size_t a3 = mark();
    span(1, a0, a1);
    span(2, a1, a2);
    span(3, a2, a3);
    if (err == cudaSuccess) err = cudaEventRecord(evE[l], s);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(sg, evR[l], 0);
    const size_t g0 = mark_on(sg);
    if (err == cudaSuccess) err = launch_rotate(P, LL, sg);
    size_t g1 = mark_on(sg);
    span(1, g0, g1);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(sg, evE[l], 0);
    if (err == cudaSuccess) err = launch_gemm_dense(P, LL, H.max_tiles[l], sg);
    if (err == cudaSuccess) err = launch_gemm_tiny(P, LL, sg);
    if (err == cudaSuccess && ss) {
      // the structured path on the split GEMM: SRRSC, the three segment lists and R,
      // then the near, W and apply products, then the tiles that stayed dense (FP64)
      int64_t Tmax, ldw;
      level_struct_dims(LL, H.struct_m, Tmax, ldw);
      SA.Tmax = (int)Tmax;
      SA.ldw = ldw;
      SA.status = P.status;
      SA.flops = P.stats ? &P.stats->struct_flops : nullptr;
      SA.ranks = P.stats ? P.stats->srrsc : nullptr;
      SA.fallback_only = 1;
      const int nseg = (int)(2 * LL.merges);
      const int64_t items = (int64_t)nseg * Tmax;
      SSArgs A;
      memset(&A, 0, sizeof(A));
      A.ssegs = P.segs;
      A.nseg = nseg;
      A.S = SA;
      A.digits = P.split_slices;
      A.near_segs = (GemmSeg*)(base + L.ss_segs);
      A.w_segs = A.near_segs + (H.ss_items + 1);
      A.ap_segs = A.w_segs + (H.ss_items + 1);
      A.img_segs = A.ap_segs + (H.ss_items + 1);
      A.counts = (int64_t*)(base + L.ss_counts);
      A.wcol0 = (int32_t*)(base + L.ss_wcol0);
      A.bcol = (int32_t*)(base + L.ss_bcol);
      A.wpos = (int32_t*)(base + L.ss_wpos);
      A.bcap = H.ss_wcap[l];
      A.W = (double*)(base + L.ss_w);
      A.ldw = ldw;
      A.wcap = H.ss_wcap[l];
      A.R = (double*)(base + L.ss_r);
      A.rcap = H.ss_wcap[l] * H.struct_m;
      A.cexp = (int32_t*)(base + L.ss_cexp);
      A.item = (int64_t*)(base + L.ss_item);
      A.accept = (int32_t*)(base + L.ss_accept);
      A.img_cap = P.img_cap;
      A.status = P.status;
      A.flops = P.stats ? &P.stats->split_flops : nullptr;
      A.bytes = P.stats ? &P.stats->split_bytes : nullptr;
      A.parts = P.stats ? P.stats->ss_parts : nullptr;
      P.ss_accept = A.accept;  // the plain split path below takes the parts this one leaves
      err = launch_struct_segs(P, LL, sg);
      if (err == cudaSuccess) err = launch_srrsc(P.segs, nseg, SA, sg);
      if (err == cudaSuccess) err = launch_ss_build(A, sg);
      // the parts' A images (digits only), then the near, W and apply products
      GemmSeg* lists[4] = {A.img_segs, A.near_segs, A.w_segs, A.ap_segs};
      const int64_t* cnts[4] = {A.counts + 3, A.counts + 0, A.counts + 1, A.counts + 2};
      size_t b4 = mark_on(sg);
      span(4, g1, b4);
      for (int k = 0; k < 4 && err == cudaSuccess; ++k) {
        cudaEvent_t mid = nullptr;
        if (timing) {
          cudaEventCreate(&mid);
          evs.push_back(mid);
        }
        const size_t b5 = timing ? evs.size() - 1 : 0;
        err = launch_split_list(lists[k], (int)items, cnts[k], P.split_slices, P.status, P.spin_budget, P.img,
                                P.split_chunk_steps, P.stats ? &P.stats->split_level_max : nullptr, sg, mid);
        const size_t b6 = mark_on(sg);
        span(5, b4, b5);
        span(6, b5, b6);
        b4 = b6;
      }
      g1 = b4;
    } else if (err == cudaSuccess && !H.ss && P.struct_min_K > 0 && LL.max_n >= P.struct_min_K) {
      int64_t Tmax, ldw;
      level_struct_dims(LL, H.struct_m, Tmax, ldw);
      SA.Tmax = (int)Tmax;
      SA.ldw = ldw;
      SA.status = P.status;
      SA.flops = P.stats ? &P.stats->struct_flops : nullptr;
      SA.ranks = P.stats ? P.stats->srrsc : nullptr;
      err = launch_struct_segs(P, LL, sg);
      if (err == cudaSuccess) err = launch_struct(P.segs, (int)(2 * LL.merges), SA, sg);
    }
    const size_t a4 = mark_on(sg);
    span(4, g1, a4);
    size_t a6 = a4;
    if (err == cudaSuccess && P.split_min_K > 0 && LL.max_n >= P.split_min_K) {
      // several passes on the host's bound: packed again on the device from the actual sizes
      const int npass = (int)H.split_chunks[l].size();
      if (npass > 1) err = launch_split_pack(P, LL, npass, sg);
      int pass = 0;
      for (auto& ch : H.split_chunks[l]) {
        cudaEvent_t mid = nullptr;
        if (timing) {
          cudaEventCreate(&mid);
          evs.push_back(mid);
        }
        const size_t b5 = timing ? evs.size() - 1 : 0;
        const size_t b4 = a6;
        if (err == cudaSuccess) err = launch_gemm_split(P, LL, ch.first, ch.second, npass > 1 ? pass : -1, sg, mid);
        ++pass;
        a6 = mark_on(sg);
        span(5, b4, b5);
        span(6, b5, a6);
      }
    }
    if (err == cudaSuccess) err = launch_copy_deflated(P, LL, o.sign_normalise, sg);
    span(7, a6, mark_on(sg));
    if (err == cudaSuccess) err = cudaEventRecord(evG[l], sg);
  }
  if (err == cudaSuccess && H.T > 0) err = cudaStreamWaitEvent(s, evG[0], 0);
  const size_t t8 = mark();
  if (err == cudaSuccess) err = launch_sign_and_output(P, o.sign_normalise, s);
  const size_t t9 = mark();
  span(8, t8, t9);
  span(9, t0, t9);
  if (err != cudaSuccess) {
    for (auto e2 : evs) cudaEventDestroy(e2);
    return TDC_ECUDA;
  }
  if (P.stats) {
    Stats hs;
    cudaMemcpyAsync(&hs, P.stats, sizeof(Stats), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
      for (auto e2 : evs) cudaEventDestroy(e2);
      return TDC_ECUDA;
    }
    float phase[12] = {0};
    for (auto& sp : spans) {
      float t = 0;
      if (cudaEventElapsedTime(&t, evs[sp.second.first], evs[sp.second.second]) == cudaSuccess) phase[sp.first] += t;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    memset(&g_last_stats, 0, sizeof(g_last_stats));
    g_last_stats.levels = H.T;
    for (int l = 0; l < H.T && l < TDC_MAX_LEVELS; ++l) {
      g_last_stats.n_merges[l] = (int64_t)hs.n_merges[l];
      g_last_stats.sum_n[l] = (int64_t)hs.sum_n[l];
      g_last_stats.sum_K[l] = (int64_t)hs.sum_K[l];
      g_last_stats.max_K[l] = hs.max_K[l];
      g_last_stats.n_rot[l] = (int64_t)hs.n_rot[l];
      g_last_stats.n_type1[l] = (int64_t)hs.n_type1[l];
      g_last_stats.gemm_flops[l] = (double)hs.gemm_flops[l];
    }
    g_last_stats.split_flops = (double)hs.split_flops;
    g_last_stats.split_bytes = (double)hs.split_bytes;
    g_last_stats.struct_flops = (double)hs.struct_flops;
    g_last_stats.launches = launches;
    g_last_stats.secular_handoffs = (int64_t)hs.handoffs;
    uint32_t lm = hs.split_level_max;
    float lmf;
    memcpy(&lmf, &lm, sizeof(lmf));
    g_last_stats.split_level_max = lmf / 16777216.0f;
    g_last_stats.lr_tiles = (int64_t)hs.srrsc[0];
    g_last_stats.lr_rank_sum = (int64_t)hs.srrsc[1];
    g_last_stats.lr_dense_fallbacks = (int64_t)hs.srrsc[2];
    g_last_stats.lr_rank_max = (int64_t)hs.srrsc[3];
    g_last_stats.lr_parts_structured = (int64_t)hs.ss_parts[0];
    g_last_stats.lr_parts_split = (int64_t)hs.ss_parts[1];
    g_last_stats.secular_iter_max = hs.iter_max;
    g_last_stats.secular_iter_mean = hs.iter_roots ? (double)hs.iter_sum / (double)hs.iter_roots : 0.0;
    for (int i = 0; i < 12; ++i) g_last_stats.phase_ms[i] = phase[i];
  }
  for (auto e2 : evs) cudaEventDestroy(e2);
  return TDC_OK;
}

}  // namespace tdc

using namespace tdc;

extern "C" {

void tdc_default_opts(tdc_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->leaf = 16;
  o->merge_mode = TDC_MERGE_AUTO;
  o->structured_min_K = 4096;
  o->lr_tile = 256;
  o->lr_tol = 1e-15;
  o->split_slices = 7;
  o->split_min_K = 128;
  o->max_iter = 64;
  o->sign_normalise = 1;
  o->collect_stats = 0;
  o->spin_budget = 1 << 24;
  o->split_chunk_k = 256;
}

int tdc_workspace_size(int64_t n, const tdc_opts* o, size_t* bytes) {
  tdc_opts d;
  tdc_default_opts(&d);
  if (o) d = *o;
  if (n < 0) return -1;
  if (validate_opts(&d)) return -2;
  if (!bytes) return -3;
  HostPlan H;
  build_plan(H, 1, &n, nullptr, nullptr, nullptr, d.leaf);
  plan_split(H, d);
  plan_struct(H, d);
  *bytes = layout_of(H).total;
  return TDC_OK;
}

int tdc_eig(int64_t n, const double* d, const double* e, double* lam, double* Q, int64_t ldq, void* ws,
            size_t ws_bytes, const tdc_opts* o, tdc_stream_t stream) {
  tdc_opts op;
  tdc_default_opts(&op);
  if (o) op = *o;
  if (n < 0) return -1;
  if (n == 0) return TDC_OK;
  if (!d) return -2;
  if (!e && n > 1) return -3;
  if (!lam) return -4;
  if (!Q) return -5;
  if (ldq < std::max<int64_t>(1, n)) return -6;
  if (validate_opts(&op)) return -9;
  HostPlan H;
  int64_t off = 0, ld = ldq;
  build_plan(H, 1, &n, &off, &off, &ld, op.leaf);
  plan_split(H, op);
  plan_struct(H, op);
  return run_plan(H, op, d, e, lam, Q, ws, ws_bytes, (cudaStream_t)stream);
}

int tdc_eig_batched_workspace_size(int32_t batch, const int64_t* n_host, const tdc_opts* o, size_t* bytes) {
  tdc_opts d;
  tdc_default_opts(&d);
  if (o) d = *o;
  if (batch < 0) return -1;
  if (batch > 0 && !n_host) return -2;
  if (validate_opts(&d)) return -3;
  if (!bytes) return -4;
  for (int32_t b = 0; b < batch; ++b)
    if (n_host[b] < 0) return -1000 - b;
  HostPlan H;
  build_plan(H, batch, n_host, nullptr, nullptr, nullptr, d.leaf);
  plan_split(H, d);
  plan_struct(H, d);
  *bytes = layout_of(H).total;
  return TDC_OK;
}

int tdc_eig_batched(int32_t batch, const int64_t* n_host, const int64_t* off_de_host, const int64_t* off_q_host,
                    const double* d, const double* e, double* lam, double* Q, void* ws, size_t ws_bytes,
                    const tdc_opts* o, tdc_stream_t stream) {
  tdc_opts op;
  tdc_default_opts(&op);
  if (o) op = *o;
  if (batch < 0) return -1;
  if (batch == 0) return TDC_OK;
  if (!n_host) return -2;
  if (!off_de_host) return -3;
  if (!off_q_host) return -4;
  if (!d) return -5;
  if (!e) return -6;
  if (!lam) return -7;
  if (!Q) return -8;
  if (validate_opts(&op)) return -11;
  for (int32_t b = 0; b < batch; ++b)
    if (n_host[b] < 0) return -1000 - b;
  HostPlan H;
  build_plan(H, batch, n_host, off_de_host, off_q_host, nullptr, op.leaf);
  plan_split(H, op);
  plan_struct(H, op);
  return run_plan(H, op, d, e, lam, Q, ws, ws_bytes, (cudaStream_t)stream);
}

int tdc_rank_one_workspace_size(int64_t K, size_t* bytes) {
  if (K < 0) return -1;
  if (!bytes) return -2;
  *bytes = rank_one_scratch_bytes(K) + 256;
  return TDC_OK;
}

// the FP32 pre-iteration scratch of a rank-one solve carved from 256-byte aligned memory
static void rank_one_carve(char* base, int64_t K, double*& zz, float2*& xz, float*& xlo) {
  const size_t k = (size_t)std::max<int64_t>(K, 1);
  zz = (double*)base;
  xz = (float2*)(base + align_up(sizeof(double) * k));
  xlo = (float*)(base + align_up(sizeof(double) * k) + align_up(sizeof(float2) * k));
}

int tdc_rank_one(int64_t K, const double* D, const double* z, double rho, int32_t* org, double* tau, double* zhat,
                 double* s, int32_t max_iter, void* ws, size_t ws_bytes, tdc_stream_t stream) {
  if (K < 0 || K > 0x7fffffff) return -1;
  if (K == 0) return TDC_OK;
  if (!D) return -2;
  if (!z) return -3;
  if (!(rho > 0.0)) return -4;
  if (!org) return -5;
  if (!tau) return -6;
  if (!zhat) return -7;
  if (!s) return -8;
  if (max_iter < 1) return -9;
  if (!ws || ws_bytes < rank_one_scratch_bytes(K) + 256) return TDC_ENOWS;
  int* st = begin_status((cudaStream_t)stream);
  if (!st) return TDC_ECUDA;
  double* zz;
  float2* xz;
  float* xlo;
  rank_one_carve((char*)(((uintptr_t)ws + 255) & ~(uintptr_t)255), K, zz, xz, xlo);
  cudaError_t e = launch_rank_one(D, z, K, rho, max_iter, org, tau, zhat, s, zz, xz, xlo, st, (cudaStream_t)stream);
  return e == cudaSuccess ? TDC_OK : TDC_ECUDA;
}

static int64_t cdiv64(int64_t a, int64_t b) { return (a + b - 1) / b; }

static int64_t cauchy_split_elems(int64_t m, int64_t K, int S, int64_t* a_elems) {
  const int64_t KB = cdiv64(K, kSplitBK);
  const int64_t a = cdiv64(m, kSplitBM) * KB * S * kSplitBM * kSplitBK;
  const int64_t b = cdiv64(K, kSplitBN) * KB * S * kSplitBN * kSplitBK;
  if (a_elems) *a_elems = a;
  return a + b;
}

__global__ void k_write_segs(GemmSeg s0, GemmSeg s1, GemmSeg* dst) {
  if (threadIdx.x == 0) { dst[0] = s0; dst[1] = s1; }
}

__global__ void k_iota(int32_t* a, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = (int32_t)i;
}

// Workspace of the stand-alone structured product on the split GEMM (one segment of
// m rows and K poles / roots): SRRSC scratch, the identity pole list, the three
// segment lists, W, R, scales and digit images (bounds as for an eigensolver level).
struct CauchySS {
  size_t segs, srank, spiv, sy, svr, scolpiv, iota, lists, counts, wcol0, bcol, wpos, w, r, cexp, item, accept, plain, img,
      total;
  int64_t T, wcap, img_elems;
};
static CauchySS cauchy_ss_layout(int64_t m, int64_t K, const tdc_opts& op) {
  CauchySS L;
  const int64_t mm = op.lr_tile, T = std::max<int64_t>(1, (K + mm - 1) / mm), ns = T * T, S = op.split_slices;
  L.T = T;
  L.wcap = std::max<int64_t>(kSplitBN, std::min<int64_t>(T * T * kSsRankBudget, ((int64_t)1 << 29) / std::max<int64_t>(m, 1)));
  L.img_elems = ss_img_bound(1, T, m, K, mm, L.wcap, S);
  size_t o = 0;
  L.segs = o; o = align_up(o + 2 * sizeof(GemmSeg));
  L.srank = o; o = align_up(o + sizeof(int) * ns);
  L.spiv = o; o = align_up(o + sizeof(int) * ns * kStructRmax);
  L.sy = o; o = align_up(o + sizeof(double) * ns * kStructRmax);
  L.svr = o; o = align_up(o + sizeof(double) * ns * mm);
  L.scolpiv = o; o = align_up(o + sizeof(int) * ns * mm);
  L.iota = o; o = align_up(o + sizeof(int32_t) * K);
  L.lists = o; o = align_up(o + 4 * sizeof(GemmSeg) * (T + 1));
  L.counts = o; o = align_up(o + 4 * sizeof(int64_t));
  L.wcol0 = o; o = align_up(o + sizeof(int32_t) * ns);
  L.bcol = o; o = align_up(o + sizeof(int32_t) * L.wcap);
  L.wpos = o; o = align_up(o + sizeof(int32_t) * L.wcap);
  L.w = o; o = align_up(o + sizeof(double) * L.wcap * std::max<int64_t>(m, 1));
  L.r = o; o = align_up(o + sizeof(double) * L.wcap * mm);
  L.cexp = o; o = align_up(o + sizeof(int32_t) * T * mm);
  L.item = o; o = align_up(o + sizeof(int64_t) * 6 * T);
  L.accept = o; o = align_up(o + sizeof(int32_t));
  L.plain = o; o = align_up(o + 2 * sizeof(GemmSeg));
  // the images: those of the structured products, or those of the plain split product
  // when the part is left to it
  L.img_elems = std::max(L.img_elems, cauchy_split_elems(m, K, S, nullptr));
  L.img = o; o = align_up(o + sizeof(__nv_bfloat16) * L.img_elems);
  L.total = 256 + o;
  return L;
}

int tdc_cauchy_gemm_workspace_size(int64_t m, int64_t K, int32_t mode, const tdc_opts* o, size_t* bytes) {
  tdc_opts op;
  tdc_default_opts(&op);
  if (o) op = *o;
  if (m < 0) return -1;
  if (K < 0) return -2;
  if (mode != TDC_MERGE_DENSE && mode != TDC_MERGE_SPLIT && mode != TDC_MERGE_STRUCTURED &&
      mode != TDC_MERGE_STRUCTURED_SPLIT)
    return -3;
  if (validate_opts(&op)) return -4;
  if (!bytes) return -5;
  if (mode == TDC_MERGE_STRUCTURED_SPLIT) {
    *bytes = cauchy_ss_layout(m, K, op).total;
    return TDC_OK;
  }
  if (mode == TDC_MERGE_DENSE) {
    *bytes = 256;
    return TDC_OK;
  }
  if (mode == TDC_MERGE_STRUCTURED) {
    const int64_t mm = op.lr_tile, T = (K + mm - 1) / mm, ns = T * T;
    *bytes = 256 + align_up(2 * sizeof(GemmSeg)) + align_up(sizeof(int) * ns) +
             align_up(sizeof(int) * ns * kStructRmax) + align_up(sizeof(double) * ns * kStructRmax) +
             align_up(sizeof(double) * ns * mm) + align_up(sizeof(int) * ns * mm) +
             align_up(sizeof(double) * T * kStructRmax * std::max<int64_t>(m, 1));
    return TDC_OK;
  }
  *bytes = 256 + align_up(2 * sizeof(GemmSeg)) +
           sizeof(__nv_bfloat16) * (size_t)cauchy_split_elems(m, K, op.split_slices, nullptr);
  return TDC_OK;
}

}  // extern "C"

// C = A * B for B the K x K Cauchy-like operand given by (D, org, tau, zhat, s) in one
// of the product modes (the body of tdc_cauchy_gemm and tdc_cauchy_like_gemm).  With
// cexp / eA (device, split modes of general operands) A enters as A 2^-eA and column j
// of the product is scaled back by 2^cexp[j].
static int cauchy_product(int64_t m, int64_t K, const double* A, int64_t lda, const double* D, const int32_t* org,
                          const double* tau, const double* zhat, const double* s, double* C, int64_t ldc,
                          int32_t mode, const tdc_opts& op, char* wbase, int* st, const int32_t* cexp,
                          const int32_t* eA, cudaStream_t cs) {
  GemmSeg sg;
  memset(&sg, 0, sizeof(sg));
  sg.ars = 1;
  sg.A = A; sg.lda = lda; sg.rows = (int32_t)m; sg.kk = (int32_t)K; sg.K = (int32_t)K;
  sg.D = D; sg.org = org; sg.tau = tau; sg.zhat = zhat; sg.scol = s;
  sg.C = C; sg.ldc = ldc;
  const bool scaled = eA != nullptr && (mode == TDC_MERGE_SPLIT || mode == TDC_MERGE_STRUCTURED_SPLIT);
  if (scaled) sg.cexp = cexp;
  cudaError_t err;
  if (mode == TDC_MERGE_DENSE) {
    err = launch_seg_dense(sg, cs);
  } else if (mode == TDC_MERGE_STRUCTURED_SPLIT) {
    const CauchySS L = cauchy_ss_layout(m, K, op);
    char* p = wbase;
    GemmSeg* segs = (GemmSeg*)(p + L.segs);
    int32_t* iota = (int32_t*)(p + L.iota);
    StructArgs SA;
    memset(&SA, 0, sizeof(SA));
    SA.m = op.lr_tile;
    SA.rmax = kStructRmax;
    SA.Tmax = (int)L.T;
    SA.tol = op.lr_tol;
    SA.srank = (int*)(p + L.srank);
    SA.spiv = (int*)(p + L.spiv);
    SA.sy = (double*)(p + L.sy);
    SA.svr = (double*)(p + L.svr);
    SA.scolpiv = (int*)(p + L.scolpiv);
    SA.ldw = m;
    SA.status = st;
    SA.fallback_only = 1;
    SSArgs A;
    memset(&A, 0, sizeof(A));
    A.ssegs = segs;
    A.nseg = 1;
    A.S = SA;
    A.digits = op.split_slices;
    A.near_segs = (GemmSeg*)(p + L.lists);
    A.w_segs = A.near_segs + (L.T + 1);
    A.ap_segs = A.w_segs + (L.T + 1);
    A.img_segs = A.ap_segs + (L.T + 1);
    A.counts = (int64_t*)(p + L.counts);
    A.wcol0 = (int32_t*)(p + L.wcol0);
    A.bcol = (int32_t*)(p + L.bcol);
    A.wpos = (int32_t*)(p + L.wpos);
    A.bcap = L.wcap;
    A.W = (double*)(p + L.w);
    A.ldw = m;
    A.wcap = L.wcap;
    A.R = (double*)(p + L.r);
    A.rcap = L.wcap * op.lr_tile;
    A.cexp = (int32_t*)(p + L.cexp);
    A.item = (int64_t*)(p + L.item);
    A.accept = (int32_t*)(p + L.accept);
    A.img_cap = L.img_elems;
    A.status = st;
    __nv_bfloat16* img = (__nv_bfloat16*)(p + L.img);
    sg.near_m = op.lr_tile;
    sg.plist = iota;
    GemmSeg last;
    memset(&last, 0, sizeof(last));
    k_iota<<<(unsigned)std::min<int64_t>(1024, (K + 255) / 256), 256, 0, cs>>>(iota, K);
    err = cudaGetLastError();
    if (err == cudaSuccess) {
      k_write_segs<<<1, 32, 0, cs>>>(sg, last, segs);
      err = cudaGetLastError();
    }
    if (err == cudaSuccess && scaled) err = launch_cauchy_like_patch(segs, eA, cs);
    if (err == cudaSuccess) err = launch_srrsc(segs, 1, SA, cs);
    if (err == cudaSuccess) err = launch_ss_build(A, cs);
    GemmSeg* lists[4] = {A.img_segs, A.near_segs, A.w_segs, A.ap_segs};
    const int64_t* cnts[4] = {A.counts + 3, A.counts + 0, A.counts + 1, A.counts + 2};
    for (int k = 0; k < 4 && err == cudaSuccess; ++k)
      err = launch_split_list(lists[k], (int)L.T, cnts[k], op.split_slices, st, op.spin_budget, img,
                              op.split_chunk_k / 16, nullptr, cs, nullptr);
    // the plain split product, emptied by the gate when the structured path took the part
    if (err == cudaSuccess) {
      GemmSeg* plain = (GemmSeg*)(p + L.plain);
      GemmSeg ps = sg;
      ps.near_m = 0;
      ps.plist = nullptr;
      const int64_t RT = cdiv64(m, kSplitBM), KB = cdiv64(K, kSplitBK), CT = cdiv64(K, kSplitBN);
      int64_t a_el = 0;
      const int64_t tot = cauchy_split_elems(m, K, op.split_slices, &a_el);
      ps.a_img = 0;
      ps.b_img = a_el;
      GemmSeg pl;
      memset(&pl, 0, sizeof(pl));
      pl.it_a = RT * KB;
      pl.it_b = CT * KB;
      pl.it_t = RT * CT;
      pl.a_img = tot;
      k_write_segs<<<1, 32, 0, cs>>>(ps, pl, plain);
      err = cudaGetLastError();
      if (err == cudaSuccess && scaled) err = launch_cauchy_like_patch(plain, eA, cs);
      if (err == cudaSuccess) err = launch_ss_gate(A.accept, plain, cs);
      if (err == cudaSuccess)
        err = launch_seg_split(plain, 1, op.split_slices, st, op.spin_budget, img, op.split_chunk_k / 16, cs);
    }
  } else if (mode == TDC_MERGE_STRUCTURED) {
    const int64_t mm = op.lr_tile, T = (K + mm - 1) / mm, ns = T * T;
    char* p = wbase;
    GemmSeg* segs = (GemmSeg*)p; p += align_up(2 * sizeof(GemmSeg));
    StructArgs SA;
    memset(&SA, 0, sizeof(SA));
    SA.m = (int)mm;
    SA.rmax = kStructRmax;
    SA.Tmax = (int)T;
    SA.tol = op.lr_tol;
    SA.srank = (int*)p; p += align_up(sizeof(int) * ns);
    SA.spiv = (int*)p; p += align_up(sizeof(int) * ns * kStructRmax);
    SA.sy = (double*)p; p += align_up(sizeof(double) * ns * kStructRmax);
    SA.svr = (double*)p; p += align_up(sizeof(double) * ns * mm);
    SA.scolpiv = (int*)p; p += align_up(sizeof(int) * ns * mm);
    SA.W = (double*)p;
    SA.ldw = m;
    SA.status = st;
    sg.near_m = (int32_t)mm;
    GemmSeg last;
    memset(&last, 0, sizeof(last));
    k_write_segs<<<1, 32, 0, cs>>>(sg, last, segs);
    err = cudaGetLastError();
    if (err == cudaSuccess) err = launch_seg_dense(sg, cs);  // near-diagonal tiles (written)
    if (err == cudaSuccess) err = launch_struct(segs, 1, SA, cs);  // low-rank tiles (accumulated)
  } else {
    const int S = op.split_slices;
    int64_t a_el = 0;
    const int64_t tot = cauchy_split_elems(m, K, S, &a_el);
    char* base = wbase;
    GemmSeg* segs = (GemmSeg*)base;
    __nv_bfloat16* img = (__nv_bfloat16*)(base + align_up(2 * sizeof(GemmSeg)));
    const int64_t RT = cdiv64(m, kSplitBM), KB = cdiv64(K, kSplitBK), CT = cdiv64(K, kSplitBN);
    sg.a_img = 0;
    sg.b_img = a_el;
    GemmSeg last;
    memset(&last, 0, sizeof(last));
    last.it_a = RT * KB;
    last.it_b = CT * KB;
    last.it_t = RT * CT;
    last.a_img = tot;
    k_write_segs<<<1, 32, 0, cs>>>(sg, last, segs);
    err = cudaGetLastError();
    if (err == cudaSuccess && scaled) err = launch_cauchy_like_patch(segs, eA, cs);
    if (err == cudaSuccess) err = launch_seg_split(segs, 1, S, st, op.spin_budget, img, op.split_chunk_k / 16, cs);
  }
  return err == cudaSuccess ? TDC_OK : TDC_ECUDA;
}

extern "C" {

int tdc_cauchy_gemm(int64_t m, int64_t K, const double* A, int64_t lda, const double* D, const int32_t* org,
                    const double* tau, const double* zhat, const double* s, double* C, int64_t ldc, int32_t mode,
                    const tdc_opts* o, void* ws, size_t ws_bytes, tdc_stream_t stream) {
  tdc_opts op;
  tdc_default_opts(&op);
  if (o) op = *o;
  if (m < 0 || m > 0x7fffffff) return -1;
  if (K < 0 || K > 0x7fffffff) return -2;
  if (m == 0 || K == 0) return TDC_OK;
  if (!A) return -3;
  if (lda < m) return -4;
  if (!D) return -5;
  if (!org) return -6;
  if (!tau) return -7;
  if (!zhat) return -8;
  if (!s) return -9;
  if (!C) return -10;
  if (ldc < m) return -11;
  if (mode != TDC_MERGE_DENSE && mode != TDC_MERGE_SPLIT && mode != TDC_MERGE_STRUCTURED &&
      mode != TDC_MERGE_STRUCTURED_SPLIT)
    return -12;
  if (validate_opts(&op)) return -13;
  size_t need = 0;
  tdc_cauchy_gemm_workspace_size(m, K, mode, &op, &need);
  if (!ws || ws_bytes < need) return TDC_ENOWS;
  char* wbase = (char*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
  cudaStream_t cs = (cudaStream_t)stream;
  int* st = begin_status(cs);
  if (!st) return TDC_ECUDA;
  return cauchy_product(m, K, A, lda, D, org, tau, zhat, s, C, ldc, mode, op, wbase, st, nullptr, nullptr, cs);
}

// the general Cauchy-like product: the generator arrays and scales after the product's
// own workspace
static size_t cauchy_like_extra(int64_t n) {
  return align_up(sizeof(int32_t) * n) + align_up(sizeof(double) * n) + align_up(sizeof(double) * n) +
         2 * align_up(sizeof(int32_t) * n) + 256;
}

int tdc_cauchy_like_gemm_workspace_size(int64_t m, int64_t n, int32_t mode, const tdc_opts* o, size_t* bytes) {
  if (!bytes) return -5;
  size_t b = 0;
  const int st = tdc_cauchy_gemm_workspace_size(m, n, mode, o, &b);
  if (st != TDC_OK) return st;
  *bytes = b + cauchy_like_extra(std::max<int64_t>(n, 0));
  return TDC_OK;
}

int tdc_cauchy_like_ranks_workspace_size(int64_t n, const tdc_opts* o, size_t* bytes) {
  tdc_opts op;
  tdc_default_opts(&op);
  if (o) op = *o;
  if (n < 0) return -1;
  if (validate_opts(&op)) return -2;
  if (!bytes) return -3;
  const int64_t mm = op.lr_tile, T = std::max<int64_t>(1, (n + mm - 1) / mm), ns = T * T;
  *bytes = 256 + align_up(2 * sizeof(GemmSeg)) + align_up(sizeof(int) * ns) + align_up(sizeof(int) * ns * kStructRmax) +
           align_up(sizeof(double) * ns * kStructRmax) + align_up(sizeof(double) * ns * mm) +
           align_up(sizeof(int) * ns * mm) + align_up(sizeof(int32_t) * n) + cauchy_like_extra(std::max<int64_t>(n, 0));
  return TDC_OK;
}

int tdc_cauchy_like_ranks(int64_t n, const double* d, const double* w, const double* u, const double* v,
                          const tdc_opts* o, int32_t* ranks, void* ws, size_t ws_bytes, tdc_stream_t stream) {
  tdc_opts op;
  tdc_default_opts(&op);
  if (o) op = *o;
  if (n < 0 || n > 0x7fffffff) return -1;
  if (n == 0) return TDC_OK;
  if (!d) return -2;
  if (!w) return -3;
  if (!u) return -4;
  if (!v) return -5;
  if (validate_opts(&op)) return -6;
  if (!ranks) return -7;
  size_t need = 0;
  tdc_cauchy_like_ranks_workspace_size(n, &op, &need);
  if (!ws || ws_bytes < need) return TDC_ENOWS;
  const int64_t mm = op.lr_tile, T = std::max<int64_t>(1, (n + mm - 1) / mm), ns = T * T;
  char* p = (char*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
  GemmSeg* segs = (GemmSeg*)p; p += align_up(2 * sizeof(GemmSeg));
  StructArgs SA;
  memset(&SA, 0, sizeof(SA));
  SA.m = (int)mm;
  SA.rmax = kStructRmax;
  SA.Tmax = (int)T;
  SA.tol = op.lr_tol;
  SA.all_offdiag = 1;
  SA.srank = (int*)p; p += align_up(sizeof(int) * ns);
  SA.spiv = (int*)p; p += align_up(sizeof(int) * ns * kStructRmax);
  SA.sy = (double*)p; p += align_up(sizeof(double) * ns * kStructRmax);
  SA.svr = (double*)p; p += align_up(sizeof(double) * ns * mm);
  SA.scolpiv = (int*)p; p += align_up(sizeof(int) * ns * mm);
  int32_t* iota = (int32_t*)p; p += align_up(sizeof(int32_t) * n);
  int32_t* org = (int32_t*)p; p += align_up(sizeof(int32_t) * n);
  double* tau = (double*)p; p += align_up(sizeof(double) * n);
  double* scol = (double*)p; p += align_up(sizeof(double) * n);
  int32_t* eb = (int32_t*)p;
  cudaStream_t cs = (cudaStream_t)stream;
  int* st = begin_status(cs);
  if (!st) return TDC_ECUDA;
  SA.status = st;
  if (launch_cauchy_like_prep(0, n, nullptr, 0, d, w, u, v, org, tau, scol, eb, nullptr, nullptr, nullptr, false, cs) !=
      cudaSuccess)
    return TDC_ECUDA;
  GemmSeg sg, last;
  memset(&sg, 0, sizeof(sg));
  memset(&last, 0, sizeof(last));
  sg.rows = 1;
  sg.kk = (int32_t)n;
  sg.K = (int32_t)n;
  sg.near_m = (int32_t)mm;
  sg.plist = iota;
  sg.D = d;
  sg.org = org;
  sg.tau = tau;
  sg.zhat = u;
  sg.scol = scol;
  k_iota<<<(unsigned)std::min<int64_t>(1024, (n + 255) / 256), 256, 0, cs>>>(iota, n);
  cudaError_t err = cudaGetLastError();
  if (err == cudaSuccess) {
    k_write_segs<<<1, 32, 0, cs>>>(sg, last, segs);
    err = cudaGetLastError();
  }
  if (err == cudaSuccess) err = cudaMemsetAsync(SA.srank, 0, sizeof(int) * ns, cs);
  if (err == cudaSuccess) err = launch_srrsc(segs, 1, SA, cs);
  if (err == cudaSuccess) err = cudaMemcpyAsync(ranks, SA.srank, sizeof(int32_t) * ns, cudaMemcpyDeviceToDevice, cs);
  return err == cudaSuccess ? TDC_OK : TDC_ECUDA;
}

int tdc_cauchy_like_gemm(int64_t m, int64_t n, const double* A, int64_t lda, const double* d, const double* w,
                         const double* u, const double* v, double* C, int64_t ldc, int32_t mode, const tdc_opts* o,
                         void* ws, size_t ws_bytes, tdc_stream_t stream) {
  tdc_opts op;
  tdc_default_opts(&op);
  if (o) op = *o;
  if (m < 0 || m > 0x7fffffff) return -1;
  if (n < 0 || n > 0x7fffffff) return -2;
  if (m == 0 || n == 0) return TDC_OK;
  if (!A) return -3;
  if (lda < m) return -4;
  if (!d) return -5;
  if (!w) return -6;
  if (!u) return -7;
  if (!v) return -8;
  if (!C) return -9;
  if (ldc < m) return -10;
  if (mode != TDC_MERGE_DENSE && mode != TDC_MERGE_SPLIT && mode != TDC_MERGE_STRUCTURED &&
      mode != TDC_MERGE_STRUCTURED_SPLIT)
    return -11;
  if (validate_opts(&op)) return -12;
  size_t need = 0, prod = 0;
  tdc_cauchy_like_gemm_workspace_size(m, n, mode, &op, &need);
  tdc_cauchy_gemm_workspace_size(m, n, mode, &op, &prod);
  if (!ws || ws_bytes < need) return TDC_ENOWS;
  char* wbase = (char*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
  char* x = wbase + align_up(prod);
  int32_t* org = (int32_t*)x; x += align_up(sizeof(int32_t) * n);
  double* tau = (double*)x; x += align_up(sizeof(double) * n);
  double* scol = (double*)x; x += align_up(sizeof(double) * n);
  int32_t* eb = (int32_t*)x; x += align_up(sizeof(int32_t) * n);
  int32_t* cexp = (int32_t*)x; x += align_up(sizeof(int32_t) * n);
  unsigned long long* maxsq = (unsigned long long*)x;
  int32_t* eA = (int32_t*)(x + 64);
  cudaStream_t cs = (cudaStream_t)stream;
  int* st = begin_status(cs);
  if (!st) return TDC_ECUDA;
  const bool scale = mode == TDC_MERGE_SPLIT || mode == TDC_MERGE_STRUCTURED_SPLIT;
  if (launch_cauchy_like_prep(m, n, A, lda, d, w, u, v, org, tau, scol, eb, cexp, eA, maxsq, scale, cs) != cudaSuccess)
    return TDC_ECUDA;
  return cauchy_product(m, n, A, lda, d, org, tau, u, scol, C, ldc, mode, op, wbase, st, scale ? cexp : nullptr,
                        scale ? eA : nullptr, cs);
}

// W and R (n^2 doubles each per problem), column exponents, segments and the
// digit images of the split products
static size_t adjoint_ws_bytes(int32_t batch, int64_t n) {
  return 256 + align_up(sizeof(double) * 2 * (size_t)batch * (size_t)n * (size_t)n) +
         align_up(sizeof(int32_t) * (size_t)batch * (size_t)n) + align_up(sizeof(GemmSeg) * ((size_t)batch + 1)) +
         256 + sizeof(__nv_bfloat16) * (size_t)adjoint_split_img_elems(batch, n);
}

int tdc_backward_workspace_size(int64_t n, size_t* bytes) {
  if (n < 0) return -1;
  if (!bytes) return -2;
  *bytes = adjoint_ws_bytes(1, n);
  return TDC_OK;
}

int tdc_eig_backward(int64_t n, const double* lam, const double* Q, int64_t ldq, const double* lam_bar,
                     const double* Q_bar, double* d_bar, double* e_bar, void* ws, size_t ws_bytes,
                     tdc_stream_t stream) {
  if (n < 0 || n > 0x7fffffff) return -1;
  if (n == 0) return TDC_OK;
  if (!lam) return -2;
  if (!Q) return -3;
  if (ldq < n) return -4;
  if (!d_bar) return -7;
  if (!e_bar && n > 1) return -8;
  size_t need = 0;
  tdc_backward_workspace_size(n, &need);
  if (!ws || ws_bytes < need) return TDC_ENOWS;
  double* w = (double*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
  int* st = begin_status((cudaStream_t)stream);
  if (!st) return TDC_ECUDA;
  cudaError_t e = launch_adjoint(1, (int)n, lam, Q, ldq, 0, lam_bar, Q_bar, 0, d_bar, e_bar, w, st, 1ll << 24,
                                 (cudaStream_t)stream);
  return e == cudaSuccess ? TDC_OK : TDC_ECUDA;
}

int tdc_backward_batched_workspace_size(int32_t batch, int64_t n, size_t* bytes) {
  if (batch < 0) return -1;
  if (n < 0) return -2;
  if (!bytes) return -3;
  *bytes = adjoint_ws_bytes(batch, n);
  return TDC_OK;
}

int tdc_eig_backward_batched(int32_t batch, int64_t n, const double* lam, const double* Q, const double* lam_bar,
                             const double* Q_bar, double* d_bar, double* e_bar, void* ws, size_t ws_bytes,
                             tdc_stream_t stream) {
  if (batch < 0) return -1;
  if (n < 0 || n > 0x7fffffff) return -2;
  if (batch == 0 || n == 0) return TDC_OK;
  if (!lam) return -3;
  if (!Q) return -4;
  if (!d_bar) return -7;
  if (!e_bar && n > 1) return -8;
  size_t need = 0;
  tdc_backward_batched_workspace_size(batch, n, &need);
  if (!ws || ws_bytes < need) return TDC_ENOWS;
  double* w = (double*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
  int* st = begin_status((cudaStream_t)stream);
  if (!st) return TDC_ECUDA;
  const int64_t nn = n * n;
  cudaError_t e = launch_adjoint(batch, (int)n, lam, Q, n, nn, lam_bar, Q_bar, nn, d_bar, e_bar, w, st, 1ll << 24,
                                 (cudaStream_t)stream);
  return e == cudaSuccess ? TDC_OK : TDC_ECUDA;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Dense symmetric eigenproblems (Section 4, Example 3): Householder reduction to
// tridiagonal form, the divide and conquer on T, back-transform of its eigenvectors.
// ---------------------------------------------------------------------------
namespace {

size_t take(size_t& o, size_t bytes) {
  const size_t r = o;
  o += align_up(bytes);
  return r;
}

struct TrdLayout {
  size_t V, W, Vr, Wr, x, y, ps, pvy, pw, pv, bar, Aop, Bop, cexp, wmax, segs, img, total;
};

// Reduction scratch: the panel's V and W (n x kTrdNb each, column- and row-major), the
// column and A22 v, per-block partials, the panel dots, the barrier counter, and
// (n >= kTrdSplitMin) the split update's operands and digit images for trailing orders
// up to n.
TrdLayout trd_layout(int64_t n) {
  TrdLayout L;
  size_t o = 0;
  const size_t nn = (size_t)std::max<int64_t>(n, 1);
  const bool split = n >= kTrdSplitMin;
  L.V = take(o, sizeof(double) * nn * kTrdNb);
  L.W = take(o, sizeof(double) * nn * kTrdNb);
  L.Vr = take(o, sizeof(double) * nn * kTrdNb);
  L.Wr = take(o, sizeof(double) * nn * kTrdNb);
  L.x = take(o, sizeof(double) * nn);
  L.y = take(o, sizeof(double) * nn);
  L.ps = take(o, sizeof(double) * kTrdMaxBlocks);
  L.pvy = take(o, sizeof(double) * kTrdMaxBlocks);
  L.pw = take(o, sizeof(double) * kTrdNb);
  L.pv = take(o, sizeof(double) * kTrdNb);
  L.bar = take(o, 64);
  L.Aop = take(o, split ? sizeof(double) * nn * 2 * kTrdNb : 0);
  L.Bop = take(o, split ? sizeof(double) * nn * 2 * kTrdNb : 0);
  L.cexp = take(o, split ? sizeof(int32_t) * nn : 0);
  L.wmax = take(o, 64);
  L.segs = take(o, 2 * sizeof(GemmSeg));
  const int64_t KB = cdiv64(2 * kTrdNb, kSplitBK);
  const int64_t img = split ? (cdiv64(n, kSplitBM) * KB * kTrdSlices * kSplitBM * kSplitBK +
                               cdiv64(n, kSplitBN) * KB * kTrdSlices * kSplitBN * kSplitBK)
                            : 0;
  L.img = take(o, sizeof(__nv_bfloat16) * (size_t)img);
  L.total = o + 256;
  return L;
}

// split-K pieces of V^T X for a block of mb rows: enough for about kOrmTileTarget output
// tiles, at least 256 rows each
int orm_ns(int64_t mb, int64_t ncols) {
  const int64_t ct = std::max<int64_t>(1, cdiv64(ncols, kSplitBN));
  int64_t ns = cdiv64(kOrmTileTarget, ct);
  ns = std::min<int64_t>(ns, std::max<int64_t>(1, mb / 256));
  return (int)std::max<int64_t>(1, ns);
}
int64_t orm_kper(int64_t mb, int ns) { return cdiv64(cdiv64(mb, ns), kSplitBK) * kSplitBK; }

struct OrmLayout {
  size_t Vb, G, Y, Z, zexp, xexp, list1, list2, img, total;
};

OrmLayout orm_layout(int64_t n, int64_t ncols) {
  OrmLayout L;
  size_t o = 0;
  const int64_t mb = std::max<int64_t>(n - 1, 1), nc = std::max<int64_t>(ncols, 1);
  const int64_t ns = orm_ns(mb, nc), kb = kOrmKb, S = kTrdSlices;
  L.Vb = take(o, sizeof(double) * (size_t)(std::max<int64_t>(n, 1) * kb));
  L.G = take(o, sizeof(double) * (size_t)(ns * kb * kb));
  L.Y = take(o, sizeof(double) * (size_t)(ns * kb * nc));
  L.Z = take(o, sizeof(double) * (size_t)(kb * nc));
  L.zexp = take(o, sizeof(int32_t) * (size_t)nc);
  L.xexp = take(o, sizeof(int32_t) * (size_t)nc);
  L.list1 = take(o, sizeof(GemmSeg) * (size_t)(2 * ns + 1));
  L.list2 = take(o, sizeof(GemmSeg) * 2);
  // digit images of one list at a time: list 1 (A = V_b^T twice per piece, B = V_b and X),
  // list 2 (A = V_b, B = Z)
  const int64_t kt = cdiv64(mb, kSplitBK) + ns;
  const int64_t img1 =
      kt * S * (2 * kSplitBM * kSplitBK + (cdiv64(kb, kSplitBN) + cdiv64(nc, kSplitBN)) * kSplitBN * kSplitBK);
  const int64_t KB2 = cdiv64(kb, kSplitBK);
  const int64_t img2 =
      (cdiv64(mb, kSplitBM) * KB2 * kSplitBM * kSplitBK + cdiv64(nc, kSplitBN) * KB2 * kSplitBN * kSplitBK) * S;
  L.img = take(o, sizeof(__nv_bfloat16) * (size_t)std::max(img1, img2));
  L.total = o + 256;
  return L;
}

int sytrd_run(int64_t n, double* A, int64_t lda, double* d, double* e, double* tau, char* base, const tdc_opts& op,
              int* st, cudaStream_t s) {
  if (n > 2) {
    const TrdLayout L = trd_layout(n);
    if (launch_sym_fill(n, A, lda, s) != cudaSuccess) return TDC_ECUDA;
    const int grid = trd_panel_grid();
    if (grid <= 0) return TDC_ECUDA;
    TrdPanel P;
    memset(&P, 0, sizeof(P));
    P.A = A;
    P.lda = lda;
    P.n = n;
    P.V = (double*)(base + L.V);
    P.W = (double*)(base + L.W);
    P.Vr = (double*)(base + L.Vr);
    P.Wr = (double*)(base + L.Wr);
    P.d = d;
    P.e = e;
    P.tau = tau;
    P.x = (double*)(base + L.x);
    P.y = (double*)(base + L.y);
    P.ps = (double*)(base + L.ps);
    P.pvy = (double*)(base + L.pvy);
    P.pw = (double*)(base + L.pw);
    P.pv = (double*)(base + L.pv);
    P.bar = (unsigned*)(base + L.bar);
    P.status = st;
    P.budget = op.spin_budget;
    TrdUpdate U;
    memset(&U, 0, sizeof(U));
    U.A = A;
    U.lda = lda;
    U.n = n;
    U.V = P.V;
    U.W = P.W;
    U.ld = n;
    U.Aop = (double*)(base + L.Aop);
    U.Bop = (double*)(base + L.Bop);
    U.cexp = (int32_t*)(base + L.cexp);
    U.wmax = (unsigned long long*)(base + L.wmax);
    U.segs = (GemmSeg*)(base + L.segs);
    U.img = (__nv_bfloat16*)(base + L.img);
    U.status = st;
    U.budget = op.spin_budget;
    U.chunk_steps = op.split_chunk_k / 16;
    for (int64_t p = 0; p < n - 2; p += kTrdNb) {
      P.p = p;
      P.nbp = (int32_t)std::min<int64_t>(kTrdNb, n - 2 - p);
      if (launch_trd_panel(P, grid, s) != cudaSuccess) return TDC_ECUDA;
      U.t0 = p + P.nbp;
      U.nb = P.nbp;
      if (launch_trd_update(U, s) != cudaSuccess) return TDC_ECUDA;
    }
  }
  return launch_trd_tail(n, A, lda, d, e, tau, s) == cudaSuccess ? TDC_OK : TDC_ECUDA;
}

int ormtr_run(int64_t n, int64_t ncols, const double* A, int64_t lda, const double* tau, double* X, int64_t ldx,
              char* base, const tdc_opts& op, int* st, cudaStream_t s) {
  const int64_t nref = n - 2;
  if (nref <= 0 || ncols == 0) return TDC_OK;
  const OrmLayout L = orm_layout(n, ncols);
  int32_t* xexp = (int32_t*)(base + L.xexp);
  if (launch_orm_xexp(n, ncols, X, ldx, xexp, s) != cudaSuccess) return TDC_ECUDA;
  for (int64_t b = cdiv64(nref, kOrmKb) - 1; b >= 0; --b) {
    OrmStep O;
    memset(&O, 0, sizeof(O));
    O.n = n;
    O.b0 = b * kOrmKb;
    O.kbp = (int32_t)std::min<int64_t>(kOrmKb, nref - O.b0);
    O.mb = n - O.b0 - 1;
    O.ncols = ncols;
    O.Vb = (double*)(base + L.Vb);
    O.ldv = n;
    O.X = X;
    O.ldx = ldx;
    O.xexp = xexp;
    O.tau = tau;
    O.G = (double*)(base + L.G);
    O.Y = (double*)(base + L.Y);
    O.Z = (double*)(base + L.Z);
    O.zexp = (int32_t*)(base + L.zexp);
    const int ns = orm_ns(O.mb, ncols);
    O.kper = orm_kper(O.mb, ns);
    O.ns = (int32_t)cdiv64(O.mb, O.kper);
    O.list1 = (GemmSeg*)(base + L.list1);
    O.list2 = (GemmSeg*)(base + L.list2);
    O.img = (__nv_bfloat16*)(base + L.img);
    O.img2 = 0;
    O.S = kTrdSlices;
    O.status = st;
    O.budget = op.spin_budget;
    O.chunk_steps = op.split_chunk_k / 16;
    if (launch_orm_step(O, A, lda, s) != cudaSuccess) return TDC_ECUDA;
  }
  return TDC_OK;
}

// d, e, tau and 256 bytes for the range guard's maximum and exponent
size_t syevd_vec_bytes(int64_t n) { return 3 * align_up(sizeof(double) * (size_t)std::max<int64_t>(n, 1)) + 256; }

// ---- symmetric band eigenproblem: divide and conquer with b rank-one merges per node
struct BandNode {
  int64_t lo, hi;
};

int64_t band_leafmax(int64_t b) { return std::max<int64_t>(128, 8 * b); }

// nodes in post order (children before their parent); leaves have at most leafmax rows
void band_nodes(int64_t lo, int64_t hi, int64_t leafmax, std::vector<BandNode>& out) {
  if (hi - lo > leafmax) {
    const int64_t m = lo + (hi - lo) / 2;
    band_nodes(lo, m, leafmax, out);
    band_nodes(m, hi, leafmax, out);
  }
  out.push_back({lo, hi});
}

struct BandLayout {
  size_t ABw, wv, Ab, Zb, dl, el, taul, Dcur, z, Ds, zs, perm, kept, defl, rotp, rotcs, cnt, DK, zK, Dd, org, tau, zhat,
      scol, iota, Qw, prod, leafws, r1, total;
  size_t leafws_bytes;
};

// sizes of the leaves (post order) and their first rows
void band_leaves(const std::vector<BandNode>& nodes, int64_t leafmax, std::vector<int64_t>& lo,
                 std::vector<int64_t>& sz) {
  for (const BandNode& nd : nodes)
    if (nd.hi - nd.lo <= leafmax) {
      lo.push_back(nd.lo);
      sz.push_back(nd.hi - nd.lo);
    }
}

BandLayout band_layout(int64_t n, int64_t b, const tdc_opts& op) {
  BandLayout L;
  size_t o = 0;
  const size_t nn = (size_t)std::max<int64_t>(n, 1);
  const int64_t lm = std::min<int64_t>(std::max<int64_t>(n, 1), band_leafmax(b));
  std::vector<BandNode> nodes;
  band_nodes(0, std::max<int64_t>(n, 1), band_leafmax(b), nodes);
  L.ABw = take(o, sizeof(double) * (size_t)(b + 1) * nn);
  L.wv = take(o, sizeof(double) * nodes.size() * (size_t)std::max<int64_t>(b, 1) * (size_t)(b + 1));
  L.Ab = take(o, sizeof(double) * nn * (size_t)lm);
  L.Zb = take(o, sizeof(double) * nn * (size_t)lm);
  L.dl = take(o, sizeof(double) * nn);
  L.el = take(o, sizeof(double) * nn);
  L.taul = take(o, sizeof(double) * nn);
  L.Dcur = take(o, sizeof(double) * nn);
  L.z = take(o, sizeof(double) * nn);
  L.Ds = take(o, sizeof(double) * nn);
  L.zs = take(o, sizeof(double) * nn);
  L.perm = take(o, sizeof(int32_t) * nn);
  L.kept = take(o, sizeof(int32_t) * nn);
  L.defl = take(o, sizeof(int32_t) * nn);
  L.rotp = take(o, 2 * sizeof(int32_t) * nn);
  L.rotcs = take(o, 2 * sizeof(double) * nn);
  L.cnt = take(o, 64);
  L.DK = take(o, sizeof(double) * nn);
  L.zK = take(o, sizeof(double) * nn);
  L.Dd = take(o, sizeof(double) * nn);
  L.org = take(o, sizeof(int32_t) * nn);
  L.tau = take(o, sizeof(double) * nn);
  L.zhat = take(o, sizeof(double) * nn);
  L.scol = take(o, sizeof(double) * nn);
  L.iota = take(o, sizeof(int32_t) * nn);
  L.r1 = take(o, rank_one_scratch_bytes((int64_t)nn));
  L.Qw = take(o, sizeof(double) * nn * nn);
  size_t pb = 0;
  tdc_cauchy_gemm_workspace_size((int64_t)nn, (int64_t)nn, TDC_MERGE_SPLIT, &op, &pb);
  L.prod = take(o, pb);
  std::vector<int64_t> llo, lsz;
  band_leaves(nodes, band_leafmax(b), llo, lsz);
  size_t we = 0;
  tdc_eig_batched_workspace_size((int32_t)lsz.size(), lsz.data(), &op, &we);
  L.leafws_bytes = we + 256;
  L.leafws = take(o, L.leafws_bytes);
  L.total = o + 256;
  return L;
}

int sbevd_run(int64_t n, int64_t b, const double* AB, int64_t ldab, double* lam, double* Q, int64_t ldq, char* base,
              const tdc_opts& op, int* st, cudaStream_t cs) {
  const BandLayout L = band_layout(n, b, op);
  const int64_t ldw = b + 1;
  double* ABw = (double*)(base + L.ABw);
  double* wv = (double*)(base + L.wv);
  double* Dcur = (double*)(base + L.Dcur);
  double* z = (double*)(base + L.z);
  double* Ds = (double*)(base + L.Ds);
  double* zs = (double*)(base + L.zs);
  int32_t* perm = (int32_t*)(base + L.perm);
  int32_t* kept = (int32_t*)(base + L.kept);
  int32_t* defl = (int32_t*)(base + L.defl);
  int32_t* rotp = (int32_t*)(base + L.rotp);
  double* rotcs = (double*)(base + L.rotcs);
  int32_t* cnt = (int32_t*)(base + L.cnt);
  double* rhod = (double*)(base + L.cnt + 32);
  double* DK = (double*)(base + L.DK);
  double* zK = (double*)(base + L.zK);
  double* Dd = (double*)(base + L.Dd);
  int32_t* org = (int32_t*)(base + L.org);
  double* tau = (double*)(base + L.tau);
  double* zhat = (double*)(base + L.zhat);
  double* scol = (double*)(base + L.scol);
  int32_t* iota = (int32_t*)(base + L.iota);
  double* Qw = (double*)(base + L.Qw);
  char* prod = base + L.prod;
  std::vector<BandNode> nodes;
  band_nodes(0, n, band_leafmax(b), nodes);
  // scratch of the sort and the deflation: arrays that the gather, the secular solve and
  // the product write only after them
  BdScratch S;
  S.sk = DK;
  S.si = org;
  S.surv = org;
  S.slot = (int32_t*)zK;
  S.c = tau;
  S.s = zhat;
  S.w = DK;
  S.dp = scol;
  S.dn = Dd;
  if (launch_bd_copy_band(n, (int)b, AB, ldab, ABw, cs) != cudaSuccess) return TDC_ECUDA;
  // entries outside [2^-400, 2^400]: the band copy scaled by a power of two
  unsigned long long* rmx = (unsigned long long*)(base + L.cnt + 40);
  int* res = (int*)(base + L.cnt + 48);
  if (launch_range_scale(ABw, ldw, n, ldw, 0, rmx, res, cs) != cudaSuccess) return TDC_ECUDA;
  if (launch_bd_zero(n, n, Q, ldq, cs) != cudaSuccess) return TDC_ECUDA;
  k_iota<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, cs>>>(iota, n);
  // tearings (they touch disjoint entries: nodes have at least 4b rows)
  for (size_t i = 0; i < nodes.size(); ++i) {
    const BandNode& nd = nodes[i];
    if (nd.hi - nd.lo <= band_leafmax(b)) continue;
    const int64_t m = nd.lo + (nd.hi - nd.lo) / 2;
    if (launch_bd_tear(ABw, ldw, (int)b, m, wv + i * b * (b + 1), cs) != cudaSuccess) return TDC_ECUDA;
  }
  // leaves, all at once: dense blocks of the torn band reduced to tridiagonal form (a block
  // each), their tridiagonals solved as one batch, the eigenvectors back-transformed into Q
  {
    const int64_t lm = std::min<int64_t>(n, band_leafmax(b));
    std::vector<int64_t> llo, lsz;
    band_leaves(nodes, band_leafmax(b), llo, lsz);
    BdLeafArgs A;
    memset(&A, 0, sizeof(A));
    A.ABw = ABw;
    A.ldab = ldw;
    A.b = (int32_t)b;
    A.lmax = lm;
    A.Ab = (double*)(base + L.Ab);
    A.d = (double*)(base + L.dl);
    A.e = (double*)(base + L.el);
    A.tau = (double*)(base + L.taul);
    A.Zb = (double*)(base + L.Zb);
    A.Q = Q;
    A.ldq = ldq;
    std::unique_ptr<BdLeafTable> T(new BdLeafTable);  // the kernel-parameter table (copied at launch)
    for (int pass = 0; pass < 2; ++pass) {
      for (size_t c0 = 0; c0 < llo.size(); c0 += kBdLeafChunk) {
        A.nleaf = (int32_t)std::min<size_t>(kBdLeafChunk, llo.size() - c0);
        for (int32_t t = 0; t < A.nleaf; ++t) {
          T->lo[t] = llo[c0 + t];
          T->L[t] = (int32_t)lsz[c0 + t];
        }
        const cudaError_t e = pass == 0 ? launch_bd_leaf_trd(A, *T, cs) : launch_bd_leaf_back(A, *T, cs);
        if (e != cudaSuccess) return TDC_ECUDA;
      }
      if (pass == 0) {
        std::vector<int64_t> oq(llo.size());
        for (size_t t = 0; t < llo.size(); ++t) oq[t] = llo[t] * lm;
        const int r = tdc_eig_batched((int32_t)llo.size(), lsz.data(), llo.data(), oq.data(), A.d, A.e, lam,
                                      (double*)(base + L.Zb), base + L.leafws, L.leafws_bytes, &op, cs);
        if (r != TDC_OK) return r;
      }
    }
  }
  for (size_t i = 0; i < nodes.size(); ++i) {
    const BandNode& nd = nodes[i];
    const int64_t nn = nd.hi - nd.lo;
    double* Qn = Q + nd.lo + nd.lo * ldq;
    if (nn <= band_leafmax(b)) continue;  // a leaf, solved above
    const int64_t m = nd.lo + (nd.hi - nd.lo) / 2;
    if (cudaMemcpyAsync(Dcur, lam + nd.lo, sizeof(double) * nn, cudaMemcpyDeviceToDevice, cs) != cudaSuccess)
      return TDC_ECUDA;
    for (int64_t k = 0; k < b; ++k) {
      const double* w = wv + i * b * (b + 1) + k * (b + 1);
      if (launch_bd_z(nn, Qn, ldq, (m - b + k) - nd.lo, m - nd.lo, (int)b, w, z, cs) != cudaSuccess) return TDC_ECUDA;
      if (launch_bd_sort(nn, Dcur, z, Ds, zs, perm, S, cs) != cudaSuccess) return TDC_ECUDA;
      if (launch_bd_deflate(nn, Ds, zs, kept, defl, rotp, rotcs, cnt, rhod, S, st, cs) != cudaSuccess)
        return TDC_ECUDA;
      int32_t hc[3] = {0, 0, 0};
      double hrho = 0.0;
      if (cudaMemcpyAsync(hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
          cudaMemcpyAsync(&hrho, rhod, sizeof(double), cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
          cudaStreamSynchronize(cs) != cudaSuccess)
        return TDC_ECUDA;
      const int K = hc[0], ndf = hc[1], nr = hc[2];
      if (launch_bd_rotate(nn, Qn, ldq, perm, rotp, rotcs, nr, st, cs) != cudaSuccess) return TDC_ECUDA;
      if (launch_bd_gather(nn, Qn, ldq, perm, kept, K, defl, ndf, Ds, zs, Qw, DK, zK, Dd, st, cs) != cudaSuccess)
        return TDC_ECUDA;
      if (K > 0) {
        double* r1zz;
        float2* r1xz;
        float* r1xlo;
        rank_one_carve(base + L.r1, K, r1zz, r1xz, r1xlo);
        if (launch_rank_one(DK, zK, K, hrho, op.max_iter, org, tau, zhat, scol, r1zz, r1xz, r1xlo, st, cs) !=
            cudaSuccess)
          return TDC_ECUDA;
        const int32_t mode = K >= 128 ? TDC_MERGE_SPLIT : TDC_MERGE_DENSE;
        char* pw = (char*)(((uintptr_t)prod + 255) & ~(uintptr_t)255);
        const int r = cauchy_product(nn, K, Qw, nn, DK, org, tau, zhat, scol, Qn, ldq, mode, op, pw, st, nullptr,
                                     nullptr, cs);
        if (r != TDC_OK) return r;
      }
      if (launch_bd_finish(nn, Qw, Qn, ldq, K, ndf, DK, org, tau, Dd, Dcur, cs) != cudaSuccess) return TDC_ECUDA;
    }
    // ascending eigenvalues and the columns in that order
    if (launch_bd_sort(nn, Dcur, nullptr, Ds, nullptr, perm, S, cs) != cudaSuccess) return TDC_ECUDA;
    if (launch_bd_gather(nn, Qn, ldq, perm, iota, (int)nn, defl, 0, Ds, Ds, Qw, DK, zK, Dd, st, cs) != cudaSuccess)
      return TDC_ECUDA;
    if (launch_bd_copy_back(nn, nn, Qw, Qn, ldq, cs) != cudaSuccess) return TDC_ECUDA;
    if (cudaMemcpyAsync(lam + nd.lo, Ds, sizeof(double) * nn, cudaMemcpyDeviceToDevice, cs) != cudaSuccess)
      return TDC_ECUDA;
  }
  return launch_range_unscale(lam, n, res, cs) == cudaSuccess ? TDC_OK : TDC_ECUDA;
}

}  // namespace

extern "C" {

int tdc_sbevd_workspace_size(int64_t n, int64_t b, const tdc_opts* o, size_t* bytes) {
  tdc_opts op;
  tdc_default_opts(&op);
  if (o) op = *o;
  if (n < 0) return -1;
  if (b < 0 || b > 64 || (n > 0 && b >= n)) return -2;
  if (validate_opts(&op)) return -3;
  if (!bytes) return -4;
  *bytes = band_layout(n, b, op).total;
  return TDC_OK;
}

int tdc_sbevd(int64_t n, int64_t b, const double* AB, int64_t ldab, double* lam, double* Q, int64_t ldq, void* ws,
              size_t ws_bytes, const tdc_opts* o, tdc_stream_t stream) {
  tdc_opts op;
  tdc_default_opts(&op);
  if (o) op = *o;
  if (n < 0) return -1;
  if (n == 0) return TDC_OK;
  if (b < 0 || b > 64 || b >= n) return -2;
  if (!AB) return -3;
  if (ldab < b + 1) return -4;
  if (!lam) return -5;
  if (!Q) return -6;
  if (ldq < n) return -7;
  if (validate_opts(&op)) return -10;
  if (!ws || ws_bytes < band_layout(n, b, op).total) return TDC_ENOWS;
  cudaStream_t cs = (cudaStream_t)stream;
  int* st = begin_status(cs);
  if (!st) return TDC_ECUDA;
  StatusNest keep;
  char* base = (char*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
  return sbevd_run(n, b, AB, ldab, lam, Q, ldq, base, op, st, cs);
}

int tdc_sytrd_workspace_size(int64_t n, size_t* bytes) {
  if (n < 0) return -1;
  if (!bytes) return -2;
  *bytes = trd_layout(n).total;
  return TDC_OK;
}

int tdc_sytrd(int64_t n, double* A, int64_t lda, double* d, double* e, double* tau, void* ws, size_t ws_bytes,
              const tdc_opts* o, tdc_stream_t stream) {
  tdc_opts op;
  tdc_default_opts(&op);
  if (o) op = *o;
  if (n < 0) return -1;
  if (n == 0) return TDC_OK;
  if (!A) return -2;
  if (lda < n || lda > kTrdMaxLd) return -3;
  if (!d) return -4;
  if (n > 1 && !e) return -5;
  if (n > 1 && !tau) return -6;
  if (validate_opts(&op)) return -9;
  if (!ws || ws_bytes < trd_layout(n).total) return TDC_ENOWS;
  cudaStream_t cs = (cudaStream_t)stream;
  int* st = begin_status(cs);
  if (!st) return TDC_ECUDA;
  char* base = (char*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
  return sytrd_run(n, A, lda, d, e, tau, base, op, st, cs);
}

int tdc_ormtr_workspace_size(int64_t n, int64_t ncols, size_t* bytes) {
  if (n < 0) return -1;
  if (ncols < 0) return -2;
  if (!bytes) return -3;
  *bytes = orm_layout(n, ncols).total;
  return TDC_OK;
}

int tdc_ormtr(int64_t n, int64_t ncols, const double* A, int64_t lda, const double* tau, double* X, int64_t ldx,
              void* ws, size_t ws_bytes, const tdc_opts* o, tdc_stream_t stream) {
  tdc_opts op;
  tdc_default_opts(&op);
  if (o) op = *o;
  if (n < 0) return -1;
  if (ncols < 0) return -2;
  if (n <= 2 || ncols == 0) return TDC_OK;
  if (!A) return -3;
  if (lda < n) return -4;
  if (!tau) return -5;
  if (!X) return -6;
  if (ldx < n) return -7;
  if (validate_opts(&op)) return -10;
  if (!ws || ws_bytes < orm_layout(n, ncols).total) return TDC_ENOWS;
  cudaStream_t cs = (cudaStream_t)stream;
  int* st = begin_status(cs);
  if (!st) return TDC_ECUDA;
  char* base = (char*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
  return ormtr_run(n, ncols, A, lda, tau, X, ldx, base, op, st, cs);
}

int tdc_syevd_workspace_size(int64_t n, const tdc_opts* o, size_t* bytes) {
  if (n < 0) return -1;
  if (!bytes) return -3;
  size_t we = 0;
  if (tdc_workspace_size(n, o, &we) != TDC_OK) return -2;
  *bytes = syevd_vec_bytes(n) + std::max(we, std::max(trd_layout(n).total, orm_layout(n, n).total)) + 256;
  return TDC_OK;
}

int tdc_syevd(int64_t n, double* A, int64_t lda, double* lam, double* Z, int64_t ldz, void* ws, size_t ws_bytes,
              const tdc_opts* o, tdc_stream_t stream) {
  tdc_opts op;
  tdc_default_opts(&op);
  if (o) op = *o;
  if (n < 0) return -1;
  if (n == 0) return TDC_OK;
  if (!A) return -2;
  if (lda < n || lda > kTrdMaxLd) return -3;
  if (!lam) return -4;
  if (!Z) return -5;
  if (ldz < n) return -6;
  if (validate_opts(&op)) return -9;
  size_t need = 0;
  tdc_syevd_workspace_size(n, &op, &need);
  if (!ws || ws_bytes < need) return TDC_ENOWS;
  cudaStream_t cs = (cudaStream_t)stream;
  int* st = begin_status(cs);
  if (!st) return TDC_ECUDA;
  StatusNest keep;
  char* base = (char*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
  const size_t vb = align_up(sizeof(double) * (size_t)n);
  double* d = (double*)base;
  double* e = (double*)(base + vb);
  double* tau = (double*)(base + 2 * vb);
  unsigned long long* rmx = (unsigned long long*)(base + 3 * vb);
  int* res = (int*)(base + 3 * vb + 8);
  char* rest = base + syevd_vec_bytes(n);
  const size_t rest_bytes = ws_bytes - (size_t)(rest - (char*)ws);
  // entries outside [2^-400, 2^400]: solved scaled by a power of two (A is destroyed anyway)
  if (launch_range_scale(A, n, n, lda, 1, rmx, res, cs) != cudaSuccess) return TDC_ECUDA;
  int r = sytrd_run(n, A, lda, d, e, tau, rest, op, st, cs);
  if (r != TDC_OK) return r;
  r = tdc_eig(n, d, e, lam, Z, ldz, rest, rest_bytes, &op, stream);
  if (r != TDC_OK) return r;
  r = ormtr_run(n, n, A, lda, tau, Z, ldz, rest, op, st, cs);
  if (r != TDC_OK) return r;
  return launch_range_unscale(lam, n, res, cs) == cudaSuccess ? TDC_OK : TDC_ECUDA;
}

// Products with a structured B given by generators (Toeplitz, Hankel, Vandermonde, the
// DFT's two real parts): B generated inside the FP64 tiles or the split product's digit
// images.
static size_t operand_extra(int64_t n) {
  return align_up(2 * sizeof(double) * (size_t)std::max<int64_t>(2 * n - 1, 1)) +
         2 * align_up(sizeof(int32_t) * (size_t)std::max<int64_t>(n, 1)) + 256;
}

static size_t operand_ws(int64_t m, int64_t n, int32_t mode, const tdc_opts& op) {
  size_t b = align_up(2 * sizeof(GemmSeg));
  if (mode == TDC_MERGE_SPLIT)
    b += align_up(sizeof(__nv_bfloat16) * (size_t)cauchy_split_elems(m, n, op.split_slices, nullptr)) +
         operand_extra(n);
  return b + 256;
}

// C = A B for B of kind 1-4 (struct_entry) from tgen (toff: Toeplitz n - 1, DFT n), at
// base (aligned) of operand_ws bytes.
static cudaError_t operand_product(int64_t m, int64_t n, const double* A, int64_t lda, int kind, const double* tgen,
                                   int64_t toff, double* C, int64_t ldc, int32_t mode, const tdc_opts& op,
                                   char* base, int* st, cudaStream_t cs) {
  GemmSeg* segs = (GemmSeg*)base;
  GemmSeg sg;
  memset(&sg, 0, sizeof(sg));
  sg.A = A;
  sg.ars = 1;
  sg.lda = lda;
  sg.rows = (int32_t)m;
  sg.kk = (int32_t)n;
  sg.K = (int32_t)n;
  sg.C = C;
  sg.ldc = ldc;
  sg.tgen = tgen;
  sg.tkind = kind;
  sg.toff = toff;
  if (mode == TDC_MERGE_DENSE) return launch_seg_dense(sg, cs);
  const int S = op.split_slices;
  int64_t a_el = 0;
  const int64_t tot = cauchy_split_elems(m, n, S, &a_el);
  char* p = base + align_up(2 * sizeof(GemmSeg));
  __nv_bfloat16* img = (__nv_bfloat16*)p;
  p += align_up(sizeof(__nv_bfloat16) * (size_t)tot);
  double* win = (double*)p;
  p += align_up(2 * sizeof(double) * (size_t)(2 * n - 1));
  int32_t* cexp = (int32_t*)p;
  p += align_up(sizeof(int32_t) * (size_t)n);
  int32_t* oexp = (int32_t*)p;
  p += align_up(sizeof(int32_t) * (size_t)n);
  unsigned long long* maxsq = (unsigned long long*)p;
  int32_t* eA = (int32_t*)(p + 64);
  cudaError_t err = launch_operand_prep(m, n, A, lda, tgen, kind, win, cexp, oexp, eA, maxsq, cs);
  const int64_t RT = cdiv64(m, kSplitBM), KB = cdiv64(n, kSplitBK), CT = cdiv64(n, kSplitBN);
  sg.cexp = cexp;
  sg.oexp = oexp;
  sg.a_img = 0;
  sg.b_img = a_el;
  GemmSeg last;
  memset(&last, 0, sizeof(last));
  last.it_a = RT * KB;
  last.it_b = CT * KB;
  last.it_t = RT * CT;
  last.a_img = tot;
  if (err == cudaSuccess) {
    k_write_segs<<<1, 32, 0, cs>>>(sg, last, segs);
    err = cudaGetLastError();
  }
  if (err == cudaSuccess) err = launch_cauchy_like_patch(segs, eA, cs);
  if (err == cudaSuccess) err = launch_seg_split(segs, 1, S, st, op.spin_budget, img, op.split_chunk_k / 16, cs);
  return err;
}

int tdc_structured_gemm_workspace_size(int64_t m, int64_t n, int32_t mode, const tdc_opts* o, size_t* bytes) {
  tdc_opts op;
  tdc_default_opts(&op);
  if (o) op = *o;
  if (m < 0 || m > 0x7fffffff) return -1;
  if (n < 0 || n > 0x7fffffff) return -2;
  if (mode != TDC_MERGE_DENSE && mode != TDC_MERGE_SPLIT) return -3;
  if (validate_opts(&op)) return -4;
  if (!bytes) return -5;
  *bytes = operand_ws(m, n, mode, op);
  return TDC_OK;
}

int tdc_structured_gemm(int64_t m, int64_t n, const double* A, int64_t lda, int32_t kind, const double* t, double* C,
                        int64_t ldc, int32_t mode, const tdc_opts* o, void* ws, size_t ws_bytes,
                        tdc_stream_t stream) {
  tdc_opts op;
  tdc_default_opts(&op);
  if (o) op = *o;
  if (m < 0 || m > 0x7fffffff) return -1;
  if (n < 0 || n > 0x7fffffff) return -2;
  if (m == 0 || n == 0) return TDC_OK;
  if (!A) return -3;
  if (lda < m) return -4;
  if (kind != TDC_TOEPLITZ && kind != TDC_HANKEL && kind != TDC_VANDERMONDE) return -5;
  if (!t) return -6;
  if (!C) return -7;
  if (ldc < m) return -8;
  if (mode != TDC_MERGE_DENSE && mode != TDC_MERGE_SPLIT) return -9;
  if (validate_opts(&op)) return -10;
  if (!ws || ws_bytes < operand_ws(m, n, mode, op)) return TDC_ENOWS;
  cudaStream_t cs = (cudaStream_t)stream;
  int* st = begin_status(cs);
  if (!st) return TDC_ECUDA;
  char* base = (char*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
  return operand_product(m, n, A, lda, kind, t, n - 1, C, ldc, mode, op, base, st, cs) == cudaSuccess ? TDC_OK
                                                                                                   : TDC_ECUDA;
}

int tdc_dft_gemm_workspace_size(int64_t m, int64_t n, int32_t mode, const tdc_opts* o, size_t* bytes) {
  const int r = tdc_structured_gemm_workspace_size(m, n, mode, o, bytes);
  if (r != TDC_OK) return r;
  *bytes += 2 * align_up(sizeof(double) * (size_t)std::max<int64_t>(n, 1));
  return TDC_OK;
}

int tdc_dft_gemm(int64_t m, int64_t n, const double* A, int64_t lda, double* Cre, double* Cim, int64_t ldc,
                 int32_t mode, const tdc_opts* o, void* ws, size_t ws_bytes, tdc_stream_t stream) {
  tdc_opts op;
  tdc_default_opts(&op);
  if (o) op = *o;
  if (m < 0 || m > 0x7fffffff) return -1;
  if (n < 0 || n > 0x7fffffff) return -2;
  if (m == 0 || n == 0) return TDC_OK;
  if (!A) return -3;
  if (lda < m) return -4;
  if (!Cre) return -5;
  if (!Cim) return -6;
  if (ldc < m) return -7;
  if (mode != TDC_MERGE_DENSE && mode != TDC_MERGE_SPLIT) return -8;
  if (validate_opts(&op)) return -9;
  size_t need = 0;
  tdc_dft_gemm_workspace_size(m, n, mode, &op, &need);
  if (!ws || ws_bytes < need) return TDC_ENOWS;
  cudaStream_t cs = (cudaStream_t)stream;
  int* st = begin_status(cs);
  if (!st) return TDC_ECUDA;
  char* base = (char*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
  const size_t tb = align_up(sizeof(double) * (size_t)n);
  double* cosv = (double*)base;
  double* msinv = (double*)(base + tb);
  char* rest = base + 2 * tb;
  cudaError_t err = launch_dft_tables(n, cosv, msinv, cs);
  if (err == cudaSuccess) err = operand_product(m, n, A, lda, 4, cosv, n, Cre, ldc, mode, op, rest, st, cs);
  if (err == cudaSuccess) err = operand_product(m, n, A, lda, 4, msinv, n, Cim, ldc, mode, op, rest, st, cs);
  return err == cudaSuccess ? TDC_OK : TDC_ECUDA;
}

// Bidiagonal SVD: the Golub-Kahan tridiagonal (order 2n), its eigenvalues and vectors,
// and the singular triplets read off the positive half.
static size_t bdsdc_head(int64_t n) {
  const size_t m = (size_t)std::max<int64_t>(2 * n, 1);
  return 3 * align_up(sizeof(double) * m) + align_up(sizeof(double) * m * m);
}

int tdc_bdsdc_workspace_size(int64_t n, const tdc_opts* o, size_t* bytes) {
  if (n < 0) return -1;
  if (!bytes) return -3;
  size_t we = 0;
  if (tdc_workspace_size(2 * n, o, &we) != TDC_OK) return -2;
  *bytes = bdsdc_head(n) + we + 256;
  return TDC_OK;
}

int tdc_bdsdc(int64_t n, const double* d, const double* e, double* sigma, double* U, int64_t ldu, double* VT,
              int64_t ldvt, void* ws, size_t ws_bytes, const tdc_opts* o, tdc_stream_t stream) {
  tdc_opts op;
  tdc_default_opts(&op);
  if (o) op = *o;
  if (n < 0) return -1;
  if (n == 0) return TDC_OK;
  if (!d) return -2;
  if (n > 1 && !e) return -3;
  if (!sigma) return -4;
  if (!U) return -5;
  if (ldu < n) return -6;
  if (!VT) return -7;
  if (ldvt < n) return -8;
  if (validate_opts(&op)) return -11;
  size_t need = 0;
  tdc_bdsdc_workspace_size(n, &op, &need);
  if (!ws || ws_bytes < need) return TDC_ENOWS;
  cudaStream_t cs = (cudaStream_t)stream;
  int* st = begin_status(cs);
  if (!st) return TDC_ECUDA;
  StatusNest keep;
  char* base = (char*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
  const size_t vb = align_up(sizeof(double) * (size_t)(2 * n));
  double* td = (double*)base;
  double* te = (double*)(base + vb);
  double* lam = (double*)(base + 2 * vb);
  double* Q = (double*)(base + 3 * vb);
  char* rest = base + bdsdc_head(n);
  const size_t rest_bytes = ws_bytes - (size_t)(rest - (char*)ws);
  if (launch_gk_build(n, d, e, td, te, cs) != cudaSuccess) return TDC_ECUDA;
  const int r = tdc_eig(2 * n, td, te, lam, Q, 2 * n, rest, rest_bytes, &op, stream);
  if (r != TDC_OK) return r;
  return launch_gk_extract(n, lam, Q, 2 * n, sigma, U, ldu, VT, ldvt, cs) == cudaSuccess ? TDC_OK : TDC_ECUDA;
}

int tdc_sync_status(tdc_stream_t stream) {
  cudaStream_t cs = (cudaStream_t)stream;
  if (cudaStreamSynchronize(cs) != cudaSuccess) return TDC_ECUDA;
  // the stream's slot (a stream no call was made on: the device's last call's)
  int* slot = stream_slot(cs, false);
  if (!slot) return TDC_OK;
  int v[2] = {0, 0}, z[2] = {0, 0};
  if (cudaMemcpy(v, slot, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return TDC_ECUDA;
  if (cudaMemcpy(slot, z, sizeof(z), cudaMemcpyHostToDevice) != cudaSuccess) return TDC_ECUDA;
  if (v[0] != 0) return v[0];
  if (v[1] & kWarnSplitLevel) return TDC_WPRECISION;
  return TDC_OK;
}

int tdc_get_stats(tdc_stats* out) {
  if (!out) return -1;
  std::lock_guard<std::mutex> lk(g_mu);
  *out = g_last_stats;
  return TDC_OK;
}

const char* tdc_strerror(int status) {
  switch (status) {
    case TDC_OK: return "success";
    case TDC_ENOWS: return "workspace missing or too small";
    case TDC_ENONFINITE: return "non-finite value";
    case TDC_ENOCONV: return "iteration did not converge within its cap";
    case TDC_ETIMEOUT: return "bounded device-side wait expired";
    case TDC_ECUDA: return "CUDA runtime error";
    case TDC_EUNSUPPORTED: return "unsupported option combination";
    case TDC_ETOOLARGE: return "problem larger than the fixed scratch of tdc_eig_noalloc";
    case TDC_WPRECISION: return "warning: a split-path level sum reached half of its exact FP32 range";
    default: return status < 0 ? "invalid argument" : "unknown status";
  }
}

}  // extern "C"
