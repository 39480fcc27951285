// tdc_structured.cu -- structured eigenvector update (Section 2.1 and 3.1 of the
// paper): the Cauchy-like Qhat of a merge is cut into m x m tiles in ascending
// pole / root order (contiguous tiles, the block-data lesson of Section 3.1.1).
// Tiles on or next to the diagonal stay dense (FP64 GEMM with generated Qhat,
// restricted to those poles); every other tile (I, J) is replaced by its SRRSC
// skeleton  Qhat(I, J) P ~= Qhat(I, T) [I  Z]  (Eq. (sid)) so that
//     C(:, J) += (Qtilde(:, I) Qhat(I, T)) [I Z] P^T,
// two thin GEMMs.  Z is never stored: like Qhat it is generated from its
// generators (Theorem 2) inside the second GEMM.
//
//   k_srrsc        one CTA per far tile: complete pivoting on |A^(k)_ij|, the
//                  search in FP32 (pivot choice only; 64x the FP64 rate), the
//                  pivot value, Theorem-1 generator updates and Theorem-2
//                  generators in FP64; stops when the pivot is <= tol * the
//                  tile's first pivot; ranks above kStructRmax fall back to dense.
//   k_struct_w     W_IJ = Qtilde(:, I) Qhat(I, pivots of (I, J))   (FP64)
//   k_struct_apply C(:, J) += sum_I W_IJ R_IJ with R_IJ = [I Z] P^T generated,
//                  or the dense tile product for fallback tiles  (FP64)
#include <float.h>

#include "tdc_common.cuh"

namespace tdc {

namespace {
constexpr int kBM = 128, kBN = 64, kBK = 16, kThreads = 256;

__device__ __forceinline__ int lower_bound_list(const int* a, int n, int x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if ((a ? a[mid] : mid) < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// list positions of the poles of row tile I
__device__ __forceinline__ void row_range(const GemmSeg& sg, int I, int m, int& qa, int& qb) {
  qa = lower_bound_list(sg.plist, sg.kk, I * m);
  qb = lower_bound_list(sg.plist, sg.kk, (I + 1) * m);
}

__device__ __forceinline__ int iabs(int x) { return x < 0 ? -x : x; }
}  // namespace

// ---------------------------------------------------------------------------
// SRRSC on one far tile.
// ---------------------------------------------------------------------------
constexpr int kMaxTile = 2048;

// kF32: pivot search in FP32 on copies of the generators (tiles up to 2048); larger
// tiles search in FP64, which fits their generators in shared memory.
template <bool kF32>
__global__ void __launch_bounds__(256) k_srrsc(const GemmSeg* segs, StructArgs S) {
  extern __shared__ double sm[];
  const int s = blockIdx.y;
  const int tile = blockIdx.x;
  const int I = tile / S.Tmax, J = tile % S.Tmax;
  const GemmSeg& sg = segs[s];
  const int m = S.m;
  if (sg.near_m == 0 || sg.K == 0) return;
  const int T = (sg.K + m - 1) / m;
  if (I >= T || J >= T || iabs(I - J) <= (S.all_offdiag ? 0 : 1)) return;
  const int64_t slot = ((int64_t)s * S.Tmax + I) * S.Tmax + J;
  int qa, qb;
  row_range(sg, I, m, qa, qb);
  const int mr = qb - qa;
  const int j0 = J * m;
  const int mc = min(m, sg.K - j0);
  const int tid = threadIdx.x;
  if (mr <= 0 || mc <= 0) {
    if (tid == 0) S.srank[slot] = 0;
    return;
  }
  // shared memory: FP64 generators and nodes, FP32 copies for the pivot search
  double* u = sm;
  double* v = u + m;
  double* dr = v + m;
  double* wo = dr + m;
  double* wt = wo + m;
  float* uf = reinterpret_cast<float*>(wt + m);
  float* vf = uf + (kF32 ? m : 0);
  float* df = vf + (kF32 ? m : 0);
  float* wf = df + (kF32 ? m : 0);
  uint8_t* ract = reinterpret_cast<uint8_t*>(wf + (kF32 ? m : 0));
  uint8_t* cact = ract + m;
  __shared__ int prow[kStructRmax], pcol[kStructRmax];
  __shared__ float redv[8];
  __shared__ int redi[8];
  __shared__ int s_piv, s_stop, s_r;
  __shared__ double s_amax0;
  for (int i = tid; i < mr; i += blockDim.x) {
    const int p = sg.plist ? sg.plist[qa + i] : qa + i;
    u[i] = sg.zhat[p];
    dr[i] = sg.D[p];
    ract[i] = 1;
  }
  for (int c = tid; c < mc; c += blockDim.x) {
    const int j = j0 + c;
    v[c] = sg.scol[j];
    wo[c] = sg.D[sg.org[j]];
    wt[c] = sg.tau[j];
    cact[c] = 1;
  }
  __syncthreads();
  const double ref = dr[0];
  if (kF32) {
    for (int i = tid; i < mr; i += blockDim.x) { df[i] = (float)(dr[i] - ref); uf[i] = (float)u[i]; }
    for (int c = tid; c < mc; c += blockDim.x) { wf[c] = (float)((wo[c] - ref) + wt[c]); vf[c] = (float)v[c]; }
  }
  if (tid == 0) { s_r = 0; s_stop = 0; s_amax0 = 0.0; }
  __syncthreads();
  bool fallback = false;
  for (;;) {
    // FP32 complete-pivoting search over the active Schur complement
    // a thread per column, the rows in order (the entry with the smallest index wins ties)
    float best = -1.0f;
    int bidx = 0x7fffffff;
    for (int c = tid; c < mc; c += blockDim.x) {
      if (!cact[c]) continue;
      if (kF32) {
        const float vc = vf[c], wc = wf[c];
        for (int i = 0; i < mr; ++i) {
          if (!ract[i]) continue;
          const float val = fabsf(uf[i] * vc) / fabsf(df[i] - wc);
          if (val > best || (val == best && i * mc + c < bidx)) { best = val; bidx = i * mc + c; }
        }
      } else {
        const double vc = v[c], woc = wo[c], wtc = wt[c];
        for (int i = 0; i < mr; ++i) {
          if (!ract[i]) continue;
          const float val = (float)(fabs(u[i] * vc) / fabs((dr[i] - woc) - wtc));
          if (val > best || (val == best && i * mc + c < bidx)) { best = val; bidx = i * mc + c; }
        }
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
      if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
    }
    if ((tid & 31) == 0) { redv[tid >> 5] = best; redi[tid >> 5] = bidx; }
    __syncthreads();
    if (tid == 0) {
      float b = redv[0];
      int bi = redi[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        if (redv[w] > b || (redv[w] == b && redi[w] < bi)) { b = redv[w]; bi = redi[w]; }
      int stop = 0;
      if (!(b > 0.0f) || bi == 0x7fffffff) {
        stop = 1;
      } else {
        const int i = bi / mc, c = bi - i * mc;
        const double a = u[i] * v[c] / ((dr[i] - wo[c]) - wt[c]);
        if (s_r == 0) s_amax0 = fabs(a);
        if (fabs(a) <= S.tol * s_amax0) stop = 1;
        else if (s_r >= S.rmax) stop = 2;
        else {
          prow[s_r] = i;
          pcol[s_r] = c;
          ract[i] = 0;
          cact[c] = 0;
          s_r += 1;
        }
      }
      s_stop = stop;
      s_piv = bi;
    }
    __syncthreads();
    if (s_stop) {
      fallback = s_stop == 2;
      break;
    }
    // Theorem 1: generators of the next Schur complement (FP64)
    const int ip = s_piv / mc, cp = s_piv - (s_piv / mc) * mc;
    const double dk = dr[ip], wko = wo[cp], wkt = wt[cp];
    for (int i = tid; i < mr; i += blockDim.x)
      if (ract[i]) {
        u[i] *= (dr[i] - dk) / ((dr[i] - wko) - wkt);
        if (kF32) uf[i] = (float)u[i];
      }
    for (int c = tid; c < mc; c += blockDim.x)
      if (cact[c]) {
        v[c] *= ((wo[c] - wko) + (wt[c] - wkt)) / ((wo[c] - dk) + wt[c]);
        if (kF32) vf[c] = (float)v[c];
      }
    __syncthreads();
  }
  const int r = s_r;
  if (S.ranks && tid == 0) {
    atomicAdd(&S.ranks[0], 1ull);
    if (fallback) atomicAdd(&S.ranks[2], 1ull);
    else {
      atomicAdd(&S.ranks[1], (unsigned long long)r);
      atomicMax(&S.ranks[3], (unsigned long long)r);
    }
  }
  if (fallback) {
    if (tid == 0) S.srank[slot] = -1;
    return;
  }
  // Theorem 2: y_a = (d_a - w_a) / v0_a * prod_{b != a} (d_b - w_a) / (w_b - w_a)
  for (int a = tid; a < r; a += blockDim.x) {
    const int ca = pcol[a];
    double y = ((dr[prow[a]] - wo[ca]) - wt[ca]) / sg.scol[j0 + ca];
    for (int b = 0; b < r; ++b) {
      if (b == a) continue;
      const int cb = pcol[b];
      y *= ((dr[prow[b]] - wo[ca]) - wt[ca]) / ((wo[cb] - wo[ca]) + (wt[cb] - wt[ca]));
    }
    S.sy[slot * S.rmax + a] = y;
    S.spiv[slot * S.rmax + a] = j0 + ca;
  }
  for (int c = tid; c < mc; c += blockDim.x) {
    int pa = -1;
    if (!cact[c])
      for (int a = 0; a < r; ++a)
        if (pcol[a] == c) pa = a;
    S.scolpiv[slot * m + c] = pa;
    S.svr[slot * m + c] = v[c];
  }
  if (tid == 0) S.srank[slot] = r;
}

// ---------------------------------------------------------------------------
// W_IJ = Qtilde(:, I) Qhat(I, pivot roots of (I, J)), r <= 64 columns.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, 2) k_struct_w(const GemmSeg* segs, StructArgs S, int J) {
  __shared__ double As[kBK][kBM];
  __shared__ double Us[kBK][kBN];
  __shared__ double sDo[kBN], sTau[kBN], sS[kBN];
  __shared__ int sCol[kBK];
  __shared__ double sDq[kBK], sZq[kBK];
  const int I = blockIdx.x, s = blockIdx.z;
  const GemmSeg& sg = segs[s];
  const int m = S.m;
  if (sg.near_m == 0 || sg.K == 0) return;
  const int T = (sg.K + m - 1) / m;
  if (I >= T || J >= T || iabs(I - J) <= 1) return;
  const int64_t slot = ((int64_t)s * S.Tmax + I) * S.Tmax + J;
  const int r = S.srank[slot];
  if (r <= 0) return;
  const int r0 = blockIdx.y * kBM;
  if (r0 >= sg.rows) return;
  int qa, qb;
  row_range(sg, I, m, qa, qb);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  if (tid < kBN) {
    if (tid < r) {
      const int piv = S.spiv[slot * S.rmax + tid];
      sDo[tid] = sg.D[sg.org[piv]];
      sTau[tid] = sg.tau[piv];
      sS[tid] = sg.scol[piv];
    } else {
      sDo[tid] = 0.0; sTau[tid] = 1.0; sS[tid] = 0.0;
    }
  }
  double acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[i][c] = 0.0;
  for (int k0 = qa; k0 < qb; k0 += kBK) {
    __syncthreads();
    if (tid < kBK) {
      const int k = k0 + tid;
      if (k < qb) {
        const int p = sg.plist ? sg.plist[k] : k;
        sCol[tid] = sg.acol ? sg.acol[p] : p;
        sDq[tid] = sg.D[p];
        sZq[tid] = sg.zhat[p];
      } else {
        sCol[tid] = -1; sDq[tid] = 0.0; sZq[tid] = 0.0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < (kBK * kBM) / kThreads; ++e) {
      const int idx = tid + e * kThreads;
      const int k = idx / kBM, rr = idx % kBM;
      const int col = sCol[k], row = r0 + rr;
      As[k][rr] = (col >= 0 && row < sg.rows) ? sg.A[row + (int64_t)col * sg.lda] : 0.0;
    }
#pragma unroll
    for (int e = 0; e < (kBK * kBN) / kThreads; ++e) {
      const int idx = tid + e * kThreads;
      const int k = idx / kBN, c = idx % kBN;
      Us[k][c] = (sZq[k] * sS[c]) * rcp_nr((sDq[k] - sDo[c]) - sTau[c]);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kBK; ++k) {
      double av[8], bv[4];
#pragma unroll
      for (int i = 0; i < 8; ++i) av[i] = As[k][ty * 8 + i];
#pragma unroll
      for (int c = 0; c < 4; ++c) bv[c] = Us[k][tx * 4 + c];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[i][c] = fma(av[i], bv[c], acc[i][c]);
    }
  }
  if (S.flops && tid == 0)
    atomicAdd(S.flops, 2ull * (unsigned long long)min(kBM, sg.rows - r0) * (unsigned long long)(qb - qa) * r);
  double* Wt = S.W + (((int64_t)s * S.Tmax + I) * S.rmax) * S.ldw;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int a = tx * 4 + c;
    if (a >= r) continue;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int row = r0 + ty * 8 + i;
      if (row < sg.rows) Wt[(int64_t)a * S.ldw + row] = acc[i][c];
    }
  }
}

// ---------------------------------------------------------------------------
// C(:, J) += sum over far tiles I of W_IJ R_IJ (R generated: unit columns at the
// pivots, Z_ab = y_a v^(r)_b / (w_a - w_b) elsewhere) or, for fallback tiles,
// Qtilde(:, I) Qhat(I, J).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, 2) k_struct_apply(const GemmSeg* segs, StructArgs S, int J) {
  __shared__ double As[kBK][kBM];
  __shared__ double Bs[kBK][kBN];
  __shared__ double sDo[kBN], sTau[kBN], sS[kBN], sVr[kBN];
  __shared__ int sPiv[kBN];
  __shared__ double sKa[kBK], sKb[kBK], sKc[kBK];
  __shared__ int sKi[kBK];
  const int s = blockIdx.z;
  const GemmSeg& sg = segs[s];
  const int m = S.m;
  if (sg.near_m == 0 || sg.K == 0) return;
  const int T = (sg.K + m - 1) / m;
  if (J >= T) return;
  const int j0 = J * m + blockIdx.y * kBN;
  if (j0 >= sg.K || blockIdx.y * kBN >= m) return;
  const int r0 = blockIdx.x * kBM;
  if (r0 >= sg.rows) return;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  if (S.fallback_only) {  // nothing to add unless a tile of this column tile stayed dense
    bool any = false;
    for (int I = 0; I < T && !any; ++I)
      any = iabs(I - J) > 1 && S.srank[((int64_t)s * S.Tmax + I) * S.Tmax + J] < 0;
    if (!any) return;
  }
  double acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[i][c] = 0.0;
  __syncthreads();
  if (tid < kBN) {
    const int j = j0 + tid;
    if (j < sg.K) { sDo[tid] = sg.D[sg.org[j]]; sTau[tid] = sg.tau[j]; sS[tid] = sg.scol[j]; }
    else { sDo[tid] = 0.0; sTau[tid] = 1.0; sS[tid] = 0.0; }
  }
  for (int I = 0; I < T; ++I) {
    if (iabs(I - J) <= 1) continue;
    const int64_t slot = ((int64_t)s * S.Tmax + I) * S.Tmax + J;
    const int r = S.srank[slot];
    if (r == 0 || (S.fallback_only && r > 0)) continue;
    __syncthreads();
    if (tid < kBN) {  // this tile's column generators for the 64 output columns
      const int c = blockIdx.y * kBN + tid;
      const bool ok = j0 + tid < sg.K;
      sPiv[tid] = (r > 0 && ok) ? S.scolpiv[slot * m + c] : -1;
      sVr[tid] = (r > 0 && ok) ? S.svr[slot * m + c] : 0.0;
    }
    int qa = 0, qb = 0;
    if (r < 0) row_range(sg, I, m, qa, qb);
    const int kn = r > 0 ? r : qb - qa;
    if (S.flops && tid == 0)
      atomicAdd(S.flops, 2ull * (unsigned long long)min(kBM, sg.rows - r0) * (unsigned long long)kn *
                             (unsigned long long)min(kBN, min(sg.K - j0, m - (int)blockIdx.y * kBN)));
    const double* Wt = S.W + (((int64_t)s * S.Tmax + I) * S.rmax) * S.ldw;
    for (int k0 = 0; k0 < kn; k0 += kBK) {
      __syncthreads();
      if (tid < kBK) {
        const int k = k0 + tid;
        if (k < kn) {
          if (r > 0) {  // pivot a: its root's nodes and y_a
            const int piv = S.spiv[slot * S.rmax + k];
            sKa[tid] = sg.D[sg.org[piv]];
            sKb[tid] = sg.tau[piv];
            sKc[tid] = S.sy[slot * S.rmax + k];
            sKi[tid] = k;
          } else {      // pole of the tile: A column and generators
            const int p = sg.plist ? sg.plist[qa + k] : qa + k;
            sKi[tid] = sg.acol ? sg.acol[p] : p;
            sKa[tid] = sg.D[p];
            sKc[tid] = sg.zhat[p];
            sKb[tid] = 0.0;
          }
        } else {
          sKi[tid] = -1; sKa[tid] = 0.0; sKb[tid] = 0.0; sKc[tid] = 0.0;
        }
      }
      __syncthreads();
#pragma unroll
      for (int e = 0; e < (kBK * kBM) / kThreads; ++e) {
        const int idx = tid + e * kThreads;
        const int k = idx / kBM, rr = idx % kBM;
        const int row = r0 + rr;
        double x = 0.0;
        if (sKi[k] >= 0 && row < sg.rows)
          x = (r > 0) ? Wt[(int64_t)sKi[k] * S.ldw + row] : sg.A[row + (int64_t)sKi[k] * sg.lda];
        As[k][rr] = x;
      }
#pragma unroll
      for (int e = 0; e < (kBK * kBN) / kThreads; ++e) {
        const int idx = tid + e * kThreads;
        const int k = idx / kBN, c = idx % kBN;
        double b = 0.0;
        if (sKi[k] >= 0 && j0 + c < sg.K) {
          if (r > 0) {
            const int pa = sPiv[c];
            if (pa == sKi[k]) b = 1.0;
            else if (pa < 0) b = sKc[k] * sVr[c] * rcp_nr((sKa[k] - sDo[c]) + (sKb[k] - sTau[c]));
          } else {
            b = (sKc[k] * sS[c]) * rcp_nr((sKa[k] - sDo[c]) - sTau[c]);
          }
        }
        Bs[k][c] = b;
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < kBK; ++k) {
        double av[8], bv[4];
#pragma unroll
        for (int i = 0; i < 8; ++i) av[i] = As[k][ty * 8 + i];
#pragma unroll
        for (int c = 0; c < 4; ++c) bv[c] = Bs[k][tx * 4 + c];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[i][c] = fma(av[i], bv[c], acc[i][c]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int j = j0 + tx * 4 + c;
    if (j >= sg.K || blockIdx.y * kBN + tx * 4 + c >= m) continue;
    const int pos = sg.cpos ? sg.cpos[j] : j;
    double* out = sg.C + (int64_t)pos * sg.ldc;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int row = r0 + ty * 8 + i;
      if (row < sg.rows) out[row] += acc[i][c];
    }
  }
}

// Segments of a tree level for the structured path: one per (merge, part); merges
// below the structured threshold get an empty segment.
__global__ void k_struct_segs(Plan P, int level, int64_t M) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= M) return;
  const Node nd = make_node(P, level, g);
  const int n = (int)(nd.hi - nd.lo), n1 = (int)(nd.mid - nd.lo);
  const int K = P.m.K[g];
  const bool use = P.struct_min_K > 0 && K >= P.struct_min_K;
  for (int p = 0; p < 2; ++p) {
    GemmSeg sg;
    memset(&sg, 0, sizeof(sg));
    sg.ars = 1;
    sg.rows = p ? n - n1 : n1;
    sg.kk = p ? P.m.nbot[g] : P.m.ntop[g];
    sg.K = use ? K : 0;
    sg.near_m = use ? P.struct_m : 0;
    sg.A = nd.src + (p ? n1 : 0);
    sg.lda = nd.lds;
    sg.acol = P.v.kept + nd.v0;
    sg.plist = (p ? P.v.blist : P.v.tlist) + nd.v0;
    sg.D = P.v.Dk + nd.v0;
    sg.org = P.v.org + nd.v0;
    sg.tau = P.v.tau + nd.v0;
    sg.zhat = P.v.zhat + nd.v0;
    sg.scol = P.v.scol + nd.v0;
    sg.C = nd.dst + (p ? n1 : 0);
    sg.ldc = nd.ldd;
    sg.cpos = P.v.posr + nd.v0;
    P.segs[2 * g + p] = sg;
  }
}

cudaError_t launch_struct_segs(const Plan& P, const LevelLaunch& L, cudaStream_t s) {
  k_struct_segs<<<(unsigned)((L.merges + 127) / 128), 128, 0, s>>>(P, L.level, L.merges);
  return cudaGetLastError();
}

// SRRSC of every far tile of nseg segments.
cudaError_t launch_srrsc(const GemmSeg* segs, int nseg, const StructArgs& A, cudaStream_t s) {
  if (nseg <= 0 || A.Tmax <= 0) return cudaSuccess;
  const bool f32 = A.m <= kMaxTile;
  const size_t smem = (size_t)A.m * (5 * sizeof(double) + (f32 ? 4 * sizeof(float) : 0) + 2);
  cudaError_t e = cudaFuncSetAttribute(f32 ? k_srrsc<true> : k_srrsc<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)(A.Tmax * A.Tmax), (unsigned)nseg);
  if (f32) k_srrsc<true><<<grid, 256, smem, s>>>(segs, A);
  else k_srrsc<false><<<grid, 256, smem, s>>>(segs, A);
  return cudaGetLastError();
}

// The tiles whose rank exceeded the cap (they stayed dense): C(:, J) += Qtilde(:, I)
// Qhat(I, J) in FP64, after the split path's products (A.fallback_only set).
cudaError_t launch_struct_fallback(const GemmSeg* segs, int nseg, const StructArgs& A, cudaStream_t s) {
  if (nseg <= 0 || A.Tmax <= 0) return cudaSuccess;
  const unsigned rt = (unsigned)((A.ldw + kBM - 1) / kBM);
  for (int J = 0; J < A.Tmax; ++J)
    k_struct_apply<<<dim3(rt, (unsigned)((A.m + kBN - 1) / kBN), (unsigned)nseg), kThreads, 0, s>>>(segs, A, J);
  return cudaGetLastError();
}

// The low-rank part for nseg segments whose dense near-diagonal part is done.
cudaError_t launch_struct(const GemmSeg* segs, int nseg, const StructArgs& A, cudaStream_t s) {
  if (nseg <= 0 || A.Tmax <= 0) return cudaSuccess;
  const int m = A.m;
  cudaError_t e = launch_srrsc(segs, nseg, A, s);
  if (e != cudaSuccess) return e;
  const unsigned rt = (unsigned)((A.ldw + kBM - 1) / kBM);
  for (int J = 0; J < A.Tmax; ++J) {
    k_struct_w<<<dim3((unsigned)A.Tmax, rt, (unsigned)nseg), kThreads, 0, s>>>(segs, A, J);
    k_struct_apply<<<dim3(rt, (unsigned)((m + kBN - 1) / kBN), (unsigned)nseg), kThreads, 0, s>>>(segs, A, J);
  }
  return cudaGetLastError();
}

}  // namespace tdc
