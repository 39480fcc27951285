// tdc_struct_split.cu -- the structured eigenvector update of Section 2.1 and
// Algorithm 2 with every product on the split-precision tensor-core GEMM.
//
// A merge part's Cauchy-like Qhat is cut into m x m tiles in ascending pole / root
// order (the FP64 structured path's tiling).  SRRSC (k_srrsc) has compressed every
// tile (I, J) with |I - J| >= 2 to its skeleton Qhat(I, J) P ~= Qhat(I, T) [I Z]
// (Eq. (sid)); here the product C = Qtilde Qhat becomes, per column tile J,
//     C(:, J) = Qtilde(:, near(J)) Qhat(near(J), J)                  near product
//             + sum_{far I} (Qtilde(:, I) Qhat(I, T_IJ)) [I Z_IJ] P^T    low rank
// and all three products run on k_gemm_split:
//   near   one segment per J over the contiguous pole range of tiles J-1..J+1,
//          written to C;
//   W      one segment per row tile I: Qtilde(:, I) times Qhat(I, pivot roots of
//          every far (I, J)), the B columns generated from a root list, the result
//          scattered into W so that the columns of each J are contiguous (W_J);
//   apply  one segment per J: W_J R_J added to C, R_J = the stacked [I Z] P^T of
//          J's far tiles, materialised in FP64 with a power-of-two scale per column
//          so that every entry is at most 1 (the split product's fixed-point range;
//          the epilogue scales the column back).
// A part is taken only when every far tile's rank stayed within the cap and its W
// columns fit the W buffer; any other part is left whole to the plain split path
// (accept[] tells its segment builder), so no tile needs a dense fallback.  Each
// taken part's A digits (Qtilde's rows over its pole list) are written once and
// read by its near and W products; |W| <= 1 by Cauchy-Schwarz on the unit rows of
// Qtilde and the unit columns of Qhat.
#include "tdc_common.cuh"

namespace tdc {

namespace {
constexpr int kBM = kSplitBM, kBN = kSplitBN, kBK = kSplitBK;
constexpr int64_t kATile = (int64_t)kBM * kBK, kBTile = (int64_t)kBN * kBK;

__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

__device__ __forceinline__ int lower_bound_i(const int* a, int n, int x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ int iabs(int x) { return x < 0 ? -x : x; }

// per (segment, tile) scratch rows of SSArgs::item
enum { kItKr = 0, kItWbase = 1, kItRofs = 2, kItKw = 3, kItBofs = 4, kItNext = 5 };

// Tiles, digit-image elements of one split segment (rows x kk times kk x K).
__device__ __forceinline__ void seg_work(const GemmSeg& g, int S, int64_t& ta, int64_t& tb, int64_t& tt,
                                         int64_t& el) {
  const int64_t RT = cdiv(g.rows, kBM), KB = cdiv(g.kk, kBK), CT = cdiv(g.K, kBN);
  ta = g.a_kt > 0 ? 0 : RT * KB;  // a segment reading a shared A image writes none
  tb = CT * KB;
  tt = (g.rows > 0 && g.K > 0) ? RT * CT : 0;
  el = ta * S * kATile + tb * S * kBTile;
}

// Work-list offsets and digit-image offsets of the first cnt segments of a list
// (one block), the terminator at [cnt]; the list's own images start at element
// `base` (a segment reading a shared A image keeps the a_img it was given); images
// beyond cap are refused.  Returns the end of the list's images (every thread).
__device__ int64_t finish_list(GemmSeg* L, int64_t cnt, int S, int64_t base, int64_t cap, int* status,
                               unsigned long long* flops, unsigned long long* bytes, int64_t (&sc)[4][32]) {
  __shared__ int64_t s_end;
  const int64_t per = (cnt + blockDim.x - 1) / blockDim.x;
  const int64_t a = min(cnt, (int64_t)threadIdx.x * per), b = min(cnt, a + per);
  int64_t v[4] = {0, 0, 0, 0};
  unsigned long long fl = 0, by = 0;
  for (int64_t i = a; i < b; ++i) {
    int64_t ta, tb, tt, el;
    seg_work(L[i], S, ta, tb, tt, el);
    v[0] += ta; v[1] += tb; v[2] += tt; v[3] += el;
    const unsigned long long r = (unsigned long long)L[i].rows, kq = (unsigned long long)L[i].kk,
                             kc = (unsigned long long)L[i].K;
    fl += 2ull * r * kq * kc;
    // algorithmic bytes: the A digits once (shared images count for their owner), the
    // B digits once, the FP64 result written (read as well when added)
    by += 2ull * S * ((L[i].a_kt > 0 ? 0ull : r * kq) + kq * kc) + (L[i].acc ? 16ull : 8ull) * r * kc;
  }
  if (flops && fl) atomicAdd(flops, fl);
  if (bytes && by) atomicAdd(bytes, by);
  block_excl_scan4(v, sc);
  for (int64_t i = a; i < b; ++i) {
    int64_t ta, tb, tt, el;
    seg_work(L[i], S, ta, tb, tt, el);
    L[i].it_a = v[0];
    L[i].it_b = v[1];
    L[i].it_t = v[2];
    if (L[i].a_kt == 0) L[i].a_img = base + v[3];
    L[i].b_img = base + v[3] + ta * S * kATile;
    v[0] += ta; v[1] += tb; v[2] += tt; v[3] += el;
  }
  if (threadIdx.x == blockDim.x - 1) {
    GemmSeg t;
    memset(&t, 0, sizeof(t));
    t.it_a = v[0];
    t.it_b = v[1];
    t.it_t = v[2];
    t.a_img = base + v[3];
    if (base + v[3] > cap) {  // cannot happen with the host's bound; never write past the images
      t.it_a = t.it_b = t.it_t = 0;
      set_status(status, TDC_EUNSUPPORTED);
    }
    L[cnt] = t;
    s_end = base + v[3];
  }
  __syncthreads();
  return s_end;
}
}  // namespace

// ---------------------------------------------------------------------------
// The three segment lists from the SRRSC results (one block of 1024 threads).
// Items are (segment s, tile t); as a column tile J = t an item owns the near and
// apply segments of J, the W columns of J's far tiles (contiguous, ordered by I)
// and the block R_J; as a row tile I = t it owns the W segment of I.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_ss_build(SSArgs A) {
  __shared__ int64_t sc[4][32];
  __shared__ int64_t tot[8];
  const StructArgs& S = A.S;
  const int m = S.m, Tm = S.Tmax, rmax = S.rmax;
  const int64_t nit = (int64_t)A.nseg * Tm;
  const int64_t per = (nit + blockDim.x - 1) / blockDim.x;
  const int64_t a0 = min(nit, (int64_t)threadIdx.x * per), a1 = min(nit, a0 + per);
  int64_t* item = A.item;
  // pass 0: which parts this path takes.  A part is taken when none of its far tiles
  // passed the rank cap and its W columns (the sum of its far tiles' ranks) fit the W
  // buffer, parts in order; every other part is left to the plain split path, so no
  // tile needs a dense fallback here.
  for (int64_t it = a0; it < a1; ++it) {
    const int s = (int)(it / Tm), t = (int)(it % Tm);
    const GemmSeg& sg = A.ssegs[s];
    const int T = (sg.near_m > 0 && sg.K > 0 && sg.rows > 0) ? (int)cdiv(sg.K, m) : 0;
    int64_t kr = 0;
    bool dense = false;
    for (int I = 0; t < T && I < T; ++I) {
      if (iabs(I - t) < 2) continue;
      const int r = S.srank[((int64_t)s * Tm + I) * Tm + t];
      if (r > 0) kr += r;
      if (r < 0) dense = true;
    }
    item[kItKr * nit + it] = dense ? -1 : kr;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t run = 0;
    unsigned long long taken = 0, left = 0;
    for (int s = 0; s < A.nseg; ++s) {
      const GemmSeg& sg = A.ssegs[s];
      const bool on = sg.near_m > 0 && sg.K > 0 && sg.rows > 0;
      int64_t tot = 0;
      bool ok = on;
      for (int t = 0; on && t < Tm; ++t) {
        const int64_t kr = item[kItKr * nit + (int64_t)s * Tm + t];
        if (kr < 0) ok = false; else tot += kr;
      }
      ok = ok && run + tot <= A.wcap;
      if (ok) run += tot;
      A.accept[s] = ok ? 1 : 0;
      if (on) { if (ok) ++taken; else ++left; }
    }
    if (A.parts) {
      atomicAdd(&A.parts[0], taken);
      atomicAdd(&A.parts[1], left);
    }
  }
  __syncthreads();
  // pass 1: per item, the W columns of J's far tiles (kr), R_J's size, and the
  // W-product columns of row tile I (kw); relative W column of each far slot
  int64_t v[4] = {0, 0, 0, 0}, w[4] = {0, 0, 0, 0};
  for (int64_t it = a0; it < a1; ++it) {
    const int s = (int)(it / Tm), t = (int)(it % Tm);
    const GemmSeg& sg = A.ssegs[s];
    const bool on = sg.near_m > 0 && sg.K > 0 && sg.rows > 0 && A.accept[s];
    const int T = on ? (int)cdiv(sg.K, m) : 0;
    int64_t kr = 0, kw = 0, mc = 0;
    if (t < T) {
      mc = min(m, sg.K - t * m);
      for (int I = 0; I < T; ++I) {
        if (iabs(I - t) < 2) continue;
        const int64_t slot = ((int64_t)s * Tm + I) * Tm + t;
        const int r = S.srank[slot];
        if (r > 0) {
          A.wcol0[slot] = (int32_t)kr;
          kr += r;
        }
      }
      for (int J = 0; J < T; ++J) {
        if (iabs(t - J) < 2) continue;
        const int r = S.srank[((int64_t)s * Tm + t) * Tm + J];
        if (r > 0) kw += r;
      }
    }
    item[kItKr * nit + it] = kr;
    item[kItKw * nit + it] = kw;
    v[0] += kr; v[1] += kr * mc; v[2] += kw; v[3] += (t < T) ? 1 : 0;
    w[0] += kr > 0 ? 1 : 0; w[1] += kw > 0 ? 1 : 0;
  }
  __syncthreads();
  int64_t vs[4] = {v[0], v[1], v[2], v[3]};
  block_excl_scan4(vs, sc);
  __syncthreads();
  int64_t ws[4] = {w[0], w[1], w[2], w[3]};
  block_excl_scan4(ws, sc);
  if (threadIdx.x == blockDim.x - 1) {
    for (int q = 0; q < 4; ++q) tot[q] = vs[q] + v[q];
    tot[4] = ws[0] + w[0];
    tot[5] = ws[1] + w[1];
  }
  __syncthreads();
  const bool fits = tot[0] <= A.wcap && tot[1] <= A.rcap && tot[2] <= A.bcap;
  if (!fits) {  // cannot happen with the host's bounds
    if (threadIdx.x == 0) {
      set_status(A.status, TDC_EUNSUPPORTED);
      A.counts[0] = A.counts[1] = A.counts[2] = 0;
      memset(&A.near_segs[0], 0, sizeof(GemmSeg));
      memset(&A.w_segs[0], 0, sizeof(GemmSeg));
      memset(&A.ap_segs[0], 0, sizeof(GemmSeg));
    }
    return;
  }
  // pass 2: offsets, absolute W columns of the far slots, near and apply segments
  int64_t wb = vs[0], rb = vs[1], bb = vs[2], ni = vs[3], ai = ws[0];
  for (int64_t it = a0; it < a1; ++it) {
    const int s = (int)(it / Tm), t = (int)(it % Tm);
    const GemmSeg& sg = A.ssegs[s];
    const bool on = sg.near_m > 0 && sg.K > 0 && sg.rows > 0 && A.accept[s];
    const int T = on ? (int)cdiv(sg.K, m) : 0;
    const int64_t kr = item[kItKr * nit + it], kw = item[kItKw * nit + it];
    item[kItWbase * nit + it] = wb;
    item[kItRofs * nit + it] = rb;
    item[kItBofs * nit + it] = bb;
    if (t < T) {
      const int j0 = t * m, mc = min(m, sg.K - j0);
      for (int I = 0; I < T; ++I) {
        if (iabs(I - t) < 2) continue;
        const int64_t slot = ((int64_t)s * Tm + I) * Tm + t;
        if (S.srank[slot] > 0) A.wcol0[slot] += (int32_t)wb;
      }
      // near product: poles of tiles t-1..t+1 (a contiguous range of the list), read
      // from the part's A image from the k-tile holding the first of them
      const int plo = t >= 1 ? (t - 1) * m : 0, phi = min(sg.K, (t + 2) * m);
      const int qa = lower_bound_i(sg.plist, sg.kk, plo), qb = lower_bound_i(sg.plist, sg.kk, phi);
      const int q0 = qa & ~(kBK - 1);
      GemmSeg g = sg;
      g.near_m = 0;
      g.plist = sg.plist + q0;
      g.kk = qb - q0;
      g.bq0 = qa - q0;
      g.a_kt = (int32_t)cdiv(sg.kk, kBK);
      g.a_img = (int64_t)(q0 / kBK) * A.digits * kATile;  // + the part image's offset (pass 4)
      g.part = s;
      g.K = mc;
      g.org = sg.org + j0;
      g.tau = sg.tau + j0;
      g.scol = sg.scol + j0;
      g.C = sg.cpos ? sg.C : sg.C + (int64_t)j0 * sg.ldc;
      g.cpos = sg.cpos ? sg.cpos + j0 : nullptr;
      g.Bd = nullptr;
      g.cexp = sg.cexp ? sg.cexp + j0 : nullptr;  // a general product's column scales
      g.bcol = nullptr;
      g.acc = 0;
      A.near_segs[ni++] = g;
      if (kr > 0) {  // apply: C(:, J) += W_J R_J
        GemmSeg h;
        memset(&h, 0, sizeof(h));
        h.ars = 1;
        h.rows = sg.rows;
        h.A = A.W + wb * A.ldw;
        h.lda = A.ldw;
        h.kk = (int32_t)kr;
        h.K = mc;
        h.Bd = A.R + rb;
        h.ldb = kr;
        h.cexp = A.cexp + ((int64_t)s * Tm + t) * m;
        h.oexp = sg.cexp ? sg.cexp + j0 : nullptr;  // R's scale in cexp, the product's here
        h.C = g.C;
        h.ldc = sg.ldc;
        h.cpos = g.cpos;
        h.acc = 1;
        A.ap_segs[ai++] = h;
      }
      wb += kr;
      rb += kr * mc;
    }
    bb += kw;
  }
  __syncthreads();
  // pass 3: the W segments and their column lists (needs every absolute W column)
  int64_t wi = ws[1];
  for (int64_t it = a0; it < a1; ++it) {
    const int s = (int)(it / Tm), t = (int)(it % Tm);
    const int64_t kw = item[kItKw * nit + it];
    if (kw == 0) continue;
    const GemmSeg& sg = A.ssegs[s];
    const int T = (int)cdiv(sg.K, m);
    const int64_t b0 = item[kItBofs * nit + it];
    int64_t k = b0;
    for (int J = 0; J < T; ++J) {
      if (iabs(t - J) < 2) continue;
      const int64_t slot = ((int64_t)s * Tm + t) * Tm + J;
      const int r = S.srank[slot];
      for (int q = 0; q < r; ++q, ++k) {
        A.bcol[k] = S.spiv[slot * rmax + q];
        A.wpos[k] = A.wcol0[slot] + q;
      }
    }
    const int qa = lower_bound_i(sg.plist, sg.kk, t * m), qb = lower_bound_i(sg.plist, sg.kk, (t + 1) * m);
    const int q0 = qa & ~(kBK - 1);
    GemmSeg g = sg;
    g.near_m = 0;
    g.plist = sg.plist + q0;
    g.kk = qb - q0;
    g.bq0 = qa - q0;
    g.a_kt = (int32_t)cdiv(sg.kk, kBK);
    g.a_img = (int64_t)(q0 / kBK) * A.digits * kATile;  // + the part image's offset (pass 4)
    g.part = s;
    g.K = (int32_t)kw;
    g.bcol = A.bcol + b0;
    g.C = A.W;
    g.ldc = A.ldw;
    g.cpos = A.wpos + b0;
    g.Bd = nullptr;
    g.cexp = nullptr;
    g.acc = 0;
    A.w_segs[wi++] = g;
  }
  // pass 4: one A image per part (written once, read by its near and W segments),
  // then the lists' own images after the shared ones; the apply products come last
  // and reuse the whole buffer
  for (int s = threadIdx.x; s < A.nseg; s += blockDim.x) {
    const GemmSeg& sg = A.ssegs[s];
    GemmSeg g;
    memset(&g, 0, sizeof(g));
    if (sg.near_m > 0 && sg.K > 0 && sg.rows > 0 && A.accept[s]) {
      g = sg;
      g.near_m = 0;
      g.K = 0;  // digits only
      g.Bd = nullptr;
      g.cexp = nullptr;
      g.bcol = nullptr;
      g.acc = 0;
      g.bq0 = 0;
      g.a_kt = 0;
    }
    A.img_segs[s] = g;
  }
  __syncthreads();
  const int64_t shared_end =
      finish_list(A.img_segs, A.nseg, A.digits, 0, A.img_cap, A.status, nullptr, A.bytes, sc);
  for (int which = 0; which < 2; ++which) {  // add each part's image offset
    GemmSeg* L = which == 0 ? A.near_segs : A.w_segs;
    const int64_t cnt = which == 0 ? tot[3] : tot[5];
    for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) L[i].a_img += A.img_segs[L[i].part].a_img;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    A.counts[0] = tot[3];
    A.counts[1] = tot[5];
    A.counts[2] = tot[4];
    A.counts[3] = A.nseg;
  }
  finish_list(A.near_segs, tot[3], A.digits, shared_end, A.img_cap, A.status, A.flops, A.bytes, sc);
  finish_list(A.w_segs, tot[5], A.digits, shared_end, A.img_cap, A.status, A.flops, A.bytes, sc);
  finish_list(A.ap_segs, tot[4], A.digits, 0, A.img_cap, A.status, A.flops, A.bytes, sc);
}

// ---------------------------------------------------------------------------
// R_J: the stacked [I Z] P^T of column tile J's far tiles, one thread per column c
// of J: the pivot row a of the column gets 1, the other pivot rows of its tile 0,
// and a column that is no pivot gets Z_ac = y_a v^(r)_c / (w_a - w_c) (Theorem 2,
// w the roots as origin + offset); the column's scale exponent makes every entry
// at most 1 in magnitude.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_ss_rmat(SSArgs A) {
  const StructArgs& S = A.S;
  const int m = S.m, Tm = S.Tmax, rmax = S.rmax;
  const int64_t nit = (int64_t)A.nseg * Tm;
  const int64_t it = blockIdx.x;
  if (it >= nit) return;
  const int64_t kr = A.item[kItKr * nit + it];
  if (kr == 0) return;
  const int s = (int)(it / Tm), J = (int)(it % Tm);
  const GemmSeg& sg = A.ssegs[s];
  const int T = (int)cdiv(sg.K, m), j0 = J * m, mc = min(m, sg.K - j0);
  const int c = blockIdx.y * blockDim.x + threadIdx.x;
  if (c >= mc) return;
  const int64_t wb = A.item[kItWbase * nit + it], rb = A.item[kItRofs * nit + it];
  const int j = j0 + c;
  const double wo = sg.D[sg.org[j]], wt = sg.tau[j];
  double* Rc = A.R + rb + (int64_t)c * kr;
  double mx = 0.0;
  for (int I = 0; I < T; ++I) {
    if (iabs(I - J) < 2) continue;
    const int64_t slot = ((int64_t)s * Tm + I) * Tm + J;
    const int r = S.srank[slot];
    if (r <= 0) continue;
    const int64_t row0 = A.wcol0[slot] - wb;
    const int pa = S.scolpiv[slot * m + c];
    const double vr = S.svr[slot * m + c];
    for (int a = 0; a < r; ++a) {
      double x;
      if (pa >= 0) {
        x = pa == a ? 1.0 : 0.0;
      } else {
        const int piv = S.spiv[slot * rmax + a];
        x = S.sy[slot * rmax + a] * vr * rcp_nr((sg.D[sg.org[piv]] - wo) + (sg.tau[piv] - wt));
      }
      Rc[row0 + a] = x;
      mx = fmax(mx, fabs(x));
    }
  }
  A.cexp[it * m + c] = mx > 1.0 ? exp_above(mx) : 0;
}

// The stand-alone product's plain split segment runs only if the structured path
// left its part: otherwise its work lists are emptied.
__global__ void k_ss_gate(const int32_t* accept, GemmSeg* plain_list) {
  if (threadIdx.x == 0 && accept[0]) plain_list[1].it_a = plain_list[1].it_b = plain_list[1].it_t = 0;
}

cudaError_t launch_ss_gate(const int32_t* accept, GemmSeg* plain_list, cudaStream_t s) {
  k_ss_gate<<<1, 32, 0, s>>>(accept, plain_list);
  return cudaGetLastError();
}

cudaError_t launch_ss_build(const SSArgs& A, cudaStream_t s) {
  if (A.nseg <= 0 || A.S.Tmax <= 0) return cudaSuccess;
  k_ss_build<<<1, 1024, 0, s>>>(A);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t nit = (int64_t)A.nseg * A.S.Tmax;
  k_ss_rmat<<<dim3((unsigned)nit, (unsigned)((A.S.m + 127) / 128)), 128, 0, s>>>(A);
  return cudaGetLastError();
}

}  // namespace tdc
