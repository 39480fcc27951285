// tdc_sytrd.cu -- dense symmetric eigenproblems around the divide and conquer: the
// Householder reduction A = Q T Q^T of a dense symmetric A to tridiagonal form and the
// back-transform X <- Q X of T's eigenvectors (Section 4, Example 3: each matrix is first
// reduced to tridiagonal form, then the tridiagonal solver runs on T).
//
// Reduction (lower triangle, blocked; Golub & Van Loan Algorithm 8.3.1 with the reflector
// convention of LAPACK's xLARFG, organised as xSYTRD / xLATRD).  Reflector k maps
// A(k+1:n, k) to beta e_1: with alpha = A(k+1, k), sigma^2 = ||A(k+2:n, k)||^2,
//   beta = -sign(alpha) sqrt(alpha^2 + sigma^2), tau = (beta - alpha) / beta,
//   v = [1, A(k+2:n, k) / (alpha - beta)]   (tau = 0, beta = alpha when sigma = 0),
// and H_k = I - tau v v^T.  Panels of kTrdNb columns.  Inside a panel column k = p + j is
// first brought up to date with the panel's earlier reflectors,
//   A(k:n, k) -= V(k:n, 0:j) W(k, 0:j)^T + W(k:n, 0:j) V(k, 0:j)^T,
// then, with A22 the trailing matrix as the panel found it,
//   y = A22 v,  pw = W^T v,  pv = V^T v,  w~ = tau (y - V pw - W pv),
//   w = w~ - (tau / 2) (w~^T v) v,  where  w~^T v = tau (v^T y - 2 pw^T pv).
// After the panel the trailing matrix takes the rank-2 nb update A22 -= V W^T + W V^T:
// on the tensor cores as a split-precision product (the merge's base-256 BF16 digits,
// exact level sums, FP64 result) once it is large, in FP64 below that.
//
// A panel is one cooperative launch (one block per SM, all resident) whose columns take
// two grid barriers each: (1) rows: finish w of the previous column, update column k,
// partial sums of sigma^2; (2) every block forms the reflector from the partials, then
// warps take the symv columns of A22 and the panel dots.  Barriers wait a bounded number
// of polls and report TDC_ETIMEOUT instead of hanging.
//
// Back-transform (compact WY): reflectors in blocks of kOrmKb, from the last block back,
//   X(b0+1:n, :) -= V T V^T X(b0+1:n, :),
// with T from the relation T^-1 = diag(1 / tau) + striu(V^T V) of Householder products,
// applied by back substitution (z_l = tau_l (y_l - sum_{i>l} G_li z_i)), which needs no
// division and leaves z_l = 0 for a tau_l = 0 reflector.  G = V^T V and Y = V^T X are
// split products cut along k into segments (partial sums added in a fixed order), then
// X += V Z with Z = -T Y is one more split product.
#include "tdc_common.cuh"

namespace tdc {

namespace {

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier of a cooperative launch: a growing arrival counter (zero before the
// launch); a block's b-th barrier waits until b * gridDim.x arrivals.  The arrival is a
// release reduction and the polls are acquire loads (a block's writes before the barrier
// are visible to every block after it).  The wait gives up after `budget` polls, records
// TDC_ETIMEOUT and returns false in the whole block.
__device__ bool grid_barrier(unsigned* ctr, unsigned& target, long long budget, int* status, int* s_flag) {
  __syncthreads();
  target += gridDim.x;
  if (threadIdx.x == 0) {
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(ctr) : "memory");
    int ok = 1;
    long long it = 0;
    while (ld_acquire_u32(ctr) < target) {
      if (++it > budget) {
        ok = 0;
        break;
      }
      if (it > 64) __nanosleep(32);
    }
    if (!ok) set_status(status, TDC_ETIMEOUT);
    *s_flag = ok;
  }
  __syncthreads();
  return *s_flag != 0;
}

// sum over a block's warps in warp order of values held by lane 0 of each warp (thread 0
// gets the result)
__device__ __forceinline__ double block_sum_lane0(double v, double* s_red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s_red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w];
  return t;
}

}  // namespace

// ---------------------------------------------------------------------------
// Reduction
// ---------------------------------------------------------------------------

// Upper triangle from the lower one (32 x 32 tiles through shared memory).
__global__ void __launch_bounds__(256) k_sym_fill(int64_t n, double* A, int64_t lda) {
  __shared__ double t[32][33];
  const int64_t T = (n + 31) / 32;
  for (int64_t b = blockIdx.x; b < T * T; b += gridDim.x) {
    const int64_t bi = b % T, bj = b / T;  // source tile (bi, bj) of the lower triangle, bi >= bj
    if (bi < bj) continue;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int r = ty; r < 32; r += 8) {
      const int64_t i = bi * 32 + r, j = bj * 32 + tx;
      t[r][tx] = (i < n && j < n) ? A[i + j * lda] : 0.0;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
      const int64_t i = bj * 32 + r, j = bi * 32 + tx;  // A(i, j) = A(j, i) for i < j
      if (i < n && j < n && i < j) A[i + j * lda] = t[tx][r];
    }
    __syncthreads();
  }
}

constexpr int kProdChunk = 16;  // columns a block takes at once in the symv

// Sums over the 32 lanes of each of C per-lane values (C a power of two <= 32): a
// reduce-scatter (every step keeps half of the values and adds the partner's other
// half), then butterflies; lanes l with l mod (32 / C) = 0 end with the sum of value
// l / (32 / C).  C = 16 takes 16 FP64 adds instead of the 80 of a butterfly per value:
// FP64 adds are scarce on this chip.
template <int C>
__device__ __forceinline__ double warp_reduce_cols(double (&v)[C]) {
  const int lane = threadIdx.x & 31;
  int o = 16;
#pragma unroll
  for (int cnt = C; cnt > 1; cnt >>= 1, o >>= 1) {
    const int half = cnt >> 1;
    const bool up = lane & o;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const double send = up ? v[i] : v[i + half], keep = up ? v[i + half] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  double r = v[0];
#pragma unroll
  for (; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  return r;
}

// Dots of nc <= C columns (base + q * stride, q < nc) with v over m rows: the block's
// threads stride over the rows, loading the next row's entries before the current row's
// multiply-adds, then reduce per column; writes y / pw / pv on threads q < nc and returns
// (thread 0) sum_q v_col(q) dot_q for the A columns.
template <int C, bool kSmem>
__device__ __forceinline__ double chunk_dots(const double* base, int64_t stride, int nc, int64_t m,
                                             const double* s_x, const double* xk, double sc, double* s_part,
                                             double* s_vy, const TrdPanel& P, int64_t k, int kind, int64_t c0) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int32_t st32 = (int32_t)stride;
  const int64_t bd = blockDim.x;
  double acc[C], cur[C];
#pragma unroll
  for (int q = 0; q < C; ++q) {
    acc[q] = 0.0;
    cur[q] = (tid < m && q < nc) ? base[tid + q * st32] : 0.0;
  }
  for (int64_t i = tid; i < m; i += bd) {
    const int64_t i2 = i + bd;
    double nxt[C];
#pragma unroll
    for (int q = 0; q < C; ++q) nxt[q] = (i2 < m && q < nc) ? base[i2 + q * st32] : 0.0;
    const double v = i == 0 ? 1.0 : (kSmem ? s_x[i] : xk[i]) * sc;
#pragma unroll
    for (int q = 0; q < C; ++q) {
      if (q < nc) acc[q] = fma(cur[q], v, acc[q]);
      cur[q] = nxt[q];
    }
  }
  constexpr int kSpan = 32 / C;
  const double r = warp_reduce_cols<C>(acc);
  if ((lane & (kSpan - 1)) == 0) s_part[warp * kProdChunk + lane / kSpan] = r;
  __syncthreads();
  if (tid < nc) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_part[w * kProdChunk + tid];
    const int64_t c = c0 + tid;  // index within its kind
    if (kind == 0) {
      P.y[k + 1 + c] = t;
      s_vy[tid] = (c == 0 ? 1.0 : (kSmem ? s_x[c] : xk[c]) * sc) * t;
    } else if (kind == 1) {
      P.pw[c] = t;
    } else {
      P.pv[c] = t;
    }
  }
  __syncthreads();
  double vy = 0.0;
  if (kind == 0 && tid == 0)
    for (int q = 0; q < nc; ++q) vy += s_vy[q];
  return vy;
}

template <bool kSmem>
__device__ __forceinline__ double chunk_dots_n(const double* base, int64_t stride, int nc, int64_t m,
                                               const double* s_x, const double* xk, double sc, double* s_part,
                                               double* s_vy, const TrdPanel& P, int64_t k, int kind, int64_t c0) {
  if (nc > 8) return chunk_dots<16, kSmem>(base, stride, nc, m, s_x, xk, sc, s_part, s_vy, P, k, kind, c0);
  if (nc > 4) return chunk_dots<8, kSmem>(base, stride, nc, m, s_x, xk, sc, s_part, s_vy, P, k, kind, c0);
  if (nc > 2) return chunk_dots<4, kSmem>(base, stride, nc, m, s_x, xk, sc, s_part, s_vy, P, k, kind, c0);
  if (nc > 1) return chunk_dots<2, kSmem>(base, stride, nc, m, s_x, xk, sc, s_part, s_vy, P, k, kind, c0);
  return chunk_dots<1, kSmem>(base, stride, nc, m, s_x, xk, sc, s_part, s_vy, P, k, kind, c0);
}

// The symv A22 v and the panel dots W^T v, V^T v as column dots over rows k+1..n-1: the m
// columns of A22 are cut into equal runs over the blocks, and so are the 2j panel
// columns (j of W, then j of V); a block takes its runs kProdChunk columns at a time.
// v_0 = 1 and v_i = x_i sc, x from the shared copy (kSmem) or from global memory.
// Returns (thread 0) the block's part of v^T A22 v.
template <bool kSmem>
__device__ double panel_products(const TrdPanel& P, int64_t k, int j, double sc, const double* s_x,
                                 double* s_part, double* s_vy) {
  const int64_t n = P.n, m = n - k - 1;
  const double* __restrict__ xk = P.x + k + 1;
  double vy = 0.0;
  {
    const int64_t per = (m + gridDim.x - 1) / gridDim.x;
    const int64_t c0 = blockIdx.x * per, c1 = c0 + per < m ? c0 + per : m;
    for (int64_t cb = c0; cb < c1; cb += kProdChunk) {
      const int nc = (int)(c1 - cb < kProdChunk ? c1 - cb : kProdChunk);
      vy += chunk_dots_n<kSmem>(P.A + (k + 1 + cb) * P.lda + k + 1, P.lda, nc, m, s_x, xk, sc, s_part, s_vy, P,
                                k, 0, cb);
    }
  }
  const int64_t items = 2 * (int64_t)j;
  if (items > 0) {
    const int64_t per = (items + gridDim.x - 1) / gridDim.x;
    const int64_t c0 = blockIdx.x * per, c1 = c0 + per < items ? c0 + per : items;
    for (int64_t cb = c0; cb < c1;) {
      const int kind = cb < j ? 1 : 2;
      const int64_t seg_end = cb < j ? j : items, lim = c1 < seg_end ? c1 : seg_end;
      const int nc = (int)(lim - cb < kProdChunk ? lim - cb : kProdChunk);
      const int64_t col = kind == 1 ? cb : cb - j;
      const double* base = (kind == 1 ? P.W : P.V) + col * n + k + 1;
      chunk_dots_n<kSmem>(base, n, nc, m, s_x, xk, sc, s_part, s_vy, P, k, kind, col);
      cb += nc;
    }
  }
  return vy;
}

// One panel: columns p .. p+nbp-1, two grid barriers per column.  Rows are taken a warp
// each, spread over the blocks (lanes over the panel columns of the row-major copies Vr,
// Wr); the symv and the panel dots go by runs of columns per block (column-major A, V,
// W), with x staged in shared memory.  Each phase issues its loads together so that a
// column costs few dependent round trips to memory.
__global__ void __launch_bounds__(kTrdThreads, 1) k_trd_panel(TrdPanel P) {
  extern __shared__ double s_x[];  // x(k+1 : n) when P.vsm
  __shared__ double s_vk[kTrdNb], s_wk[kTrdNb], s_pw[kTrdNb], s_pv[kTrdNb];
  __shared__ double s_red[kTrdThreads / 32];
  __shared__ double s_part[(kTrdThreads / 32) * kProdChunk];
  __shared__ double s_vy[kProdChunk];
  __shared__ double s_scal[8];
  __shared__ int s_flag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int kWarps = kTrdThreads / 32;
  const int64_t n = P.n, ld = P.n;
  const int64_t G = (int64_t)gridDim.x * blockDim.x, g = (int64_t)blockIdx.x * blockDim.x + tid;
  const int64_t rstep = (int64_t)gridDim.x * kWarps;  // warp-per-row stride
  unsigned target = 0;
  double* __restrict__ A = P.A;
  const int64_t lda = P.lda;
  constexpr int nb = kTrdNb;

  for (int j = 0; j < P.nbp; ++j) {
    const int64_t k = P.p + j;
    // ---- (1) finish w of column j-1, update column k with the panel so far
    double tprev = 0.0, gam = 0.0;
    // the warp's first row: its loads go out with the prelude's
    const int64_t r0 = k + blockIdx.x + (int64_t)gridDim.x * warp;
    double vrc[4] = {0.0, 0.0, 0.0, 0.0}, wrc[4] = {0.0, 0.0, 0.0, 0.0};
    double a0 = 0.0, yv0 = 0.0, vl0 = 0.0;
    if (r0 < n) {
      const double* vrow = P.Vr + r0 * nb;
      const double* wrow = P.Wr + r0 * nb;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        vrc[q] = vrow[lane + 32 * q];
        wrc[q] = wrow[lane + 32 * q];
      }
      if (lane == 0) {
        a0 = A[r0 + k * lda];
        if (j > 0) {
          yv0 = P.y[r0];
          vl0 = vrow[j - 1];
        }
      }
    }
    if (j > 0) {
      // one round trip: row k of the panel, the dots of column j-1, the partials of
      // v^T A22 v, y_k and tau_{k-1}
      for (int c = tid; c < j; c += blockDim.x) {
        s_vk[c] = P.Vr[k * nb + c];
        if (c < j - 1) {
          s_pw[c] = P.pw[c];
          s_pv[c] = P.pv[c];
          s_wk[c] = P.Wr[k * nb + c];
        }
      }
      if (warp == kWarps - 1) {
        double t = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32) t += P.pvy[b];
        t = warp_sum(t);
        if (lane == 0) {
          s_scal[4] = t;
          s_scal[5] = P.y[k];
          s_scal[6] = P.tau[k - 1];
        }
      }
      __syncthreads();
      tprev = s_scal[6];
      if (warp == 0) {
        double q = 0.0, f = 0.0;
        for (int c = lane; c < j - 1; c += 32) {
          q = fma(s_pw[c], s_pv[c], q);
          f = fma(s_vk[c], s_pw[c], fma(s_wk[c], s_pv[c], f));
        }
        q = warp_sum(q);
        f = warp_sum(f);
        if (lane == 0) {
          const double gm = tprev * (s_scal[4] - 2.0 * q);
          s_scal[0] = gm;
          s_wk[j - 1] = tprev * (s_scal[5] - f) - 0.5 * tprev * gm * s_vk[j - 1];
        }
      }
      __syncthreads();
      gam = s_scal[0];
    }
    double ss = 0.0;
    for (int64_t r = r0; r < n; r += rstep) {
      double a = a0, yv = yv0, vlast = vl0;
      if (r != r0) {  // later rows (n above the grid's warp count)
        const double* vrow = P.Vr + r * nb;
        const double* wrow = P.Wr + r * nb;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          vrc[q] = vrow[lane + 32 * q];
          wrc[q] = wrow[lane + 32 * q];
        }
        if (lane == 0) {
          a = A[r + k * lda];
          if (j > 0) {
            yv = P.y[r];
            vlast = vrow[j - 1];
          }
        }
      }
      double f = 0.0, u = 0.0;
      if (j > 1) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int c = lane + 32 * q;
          if (c < j - 1) {
            f = fma(vrc[q], s_pw[c], fma(wrc[q], s_pv[c], f));
            u = fma(vrc[q], s_wk[c], fma(wrc[q], s_vk[c], u));
          }
        }
        f = warp_sum(f);
        u = warp_sum(u);
      }
      if (lane == 0) {
        if (j > 0) {
          const double wr = (r == k) ? s_wk[j - 1] : tprev * (yv - f) - 0.5 * tprev * gam * vlast;
          P.W[r + (j - 1) * ld] = wr;
          P.Wr[r * nb + j - 1] = wr;
          u = fma(vlast, s_wk[j - 1], fma(wr, s_vk[j - 1], u));
          a -= u;
        }
        if (r == k) {
          P.d[k] = a;
          A[k + k * lda] = a;
        } else {
          P.x[r] = a;
          if (r >= k + 2) ss = fma(a, a, ss);
        }
      }
    }
    {
      const double t = block_sum_lane0(ss, s_red);
      if (tid == 0) P.ps[blockIdx.x] = t;
    }
    if (!grid_barrier(P.bar, target, P.budget, P.status, &s_flag)) return;

    // ---- (2) the reflector of column k (one round trip: the partials and x), then A22 v
    // and the panel dots
    const int64_t m = n - k - 1;
    if (P.vsm)
      for (int64_t i = tid; i < m; i += blockDim.x) s_x[i] = P.x[k + 1 + i];
    if (warp == 0) {
      const double alpha = P.x[k + 1];
      double s = 0.0;
      for (int b = lane; b < (int)gridDim.x; b += 32) s += P.ps[b];
      s = warp_sum(s);
      if (lane == 0) {
        double t = 0.0, beta = alpha, sc = 0.0;
        if (s > 0.0) {
          const double nrm = sqrt(fma(alpha, alpha, s));
          beta = -copysign(nrm, alpha);
          t = (beta - alpha) / beta;
          sc = 1.0 / (alpha - beta);
        }
        s_scal[1] = t;
        s_scal[2] = sc;
        s_scal[3] = beta;
      }
    }
    __syncthreads();
    const double sc = s_scal[2];
    if (g == 0) {
      P.tau[k] = s_scal[1];
      P.e[k] = s_scal[3];
      A[k + 1 + k * lda] = s_scal[3];
    }
    for (int64_t r = P.p + 1 + g; r < n; r += G) {
      const double v = r <= k ? 0.0 : (r == k + 1 ? 1.0 : (P.vsm ? s_x[r - k - 1] : P.x[r]) * sc);
      P.V[r + j * ld] = v;
      P.Vr[r * nb + j] = v;
      if (r >= k + 2) A[r + k * lda] = v;
    }
    const double vy = P.vsm ? panel_products<true>(P, k, j, sc, s_x, s_part, s_vy)
                            : panel_products<false>(P, k, j, sc, s_x, s_part, s_vy);
    if (tid == 0) P.pvy[blockIdx.x] = vy;
    if (!grid_barrier(P.bar, target, P.budget, P.status, &s_flag)) return;
  }

  // ---- w of the panel's last column on the trailing rows
  const int jl = P.nbp - 1;
  for (int c = tid; c < jl; c += blockDim.x) {
    s_pw[c] = P.pw[c];
    s_pv[c] = P.pv[c];
  }
  if (warp == kWarps - 1) {
    double t = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) t += P.pvy[b];
    t = warp_sum(t);
    if (lane == 0) {
      s_scal[4] = t;
      s_scal[6] = P.tau[P.p + jl];
    }
  }
  __syncthreads();
  const double tl = s_scal[6];
  if (warp == 0) {
    double q = 0.0;
    for (int c = lane; c < jl; c += 32) q = fma(s_pw[c], s_pv[c], q);
    q = warp_sum(q);
    if (lane == 0) s_scal[0] = tl * (s_scal[4] - 2.0 * q);
  }
  __syncthreads();
  const double gam = s_scal[0];
  for (int64_t r = P.p + P.nbp + blockIdx.x + (int64_t)gridDim.x * warp; r < n; r += rstep) {
    const double* vrow = P.Vr + r * nb;
    const double* wrow = P.Wr + r * nb;
    double vrc[4], wrc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      vrc[q] = vrow[lane + 32 * q];
      wrc[q] = wrow[lane + 32 * q];
    }
    double f = 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = lane + 32 * q;
      if (c < jl) f = fma(vrc[q], s_pw[c], fma(wrc[q], s_pv[c], f));
    }
    f = warp_sum(f);
    if (lane == 0) P.W[r + jl * ld] = tl * (P.y[r] - f) - 0.5 * tl * gam * vrow[jl];
  }
}

// Largest |W(t0:n, 0:nb)| as the bits of a non-negative double (zero beforehand).
__global__ void __launch_bounds__(256) k_trd_wmax(int64_t t0, int64_t n, int nb, const double* W, int64_t ld,
                                                 unsigned long long* wmax) {
  double m = 0.0;
  const int64_t rows = n - t0, total = rows * nb;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs(W[t0 + i % rows + (i / rows) * ld]));
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) atomicMax(wmax, (unsigned long long)__double_as_longlong(m));
}

// Operands of A22 -= V W^T + W V^T as one split product C += Aop Bop over K = 2 nb:
//   Aop = -[V, W 2^-ew] (m x 2nb, ld m),  Bop = [W^T; 2^ew V^T] (2nb x m, ld 2nb),
// 2^ew above every |W| so that |Aop| <= 1; column i of Bop enters scaled by 2^-cexp[i]
// (its largest entry below 1) and the product's column is scaled back.
__global__ void __launch_bounds__(256) k_trd_ops(int64_t t0, int64_t n, int nb, const double* V, const double* W,
                                                int64_t ld, const unsigned long long* wmax, double* Aop,
                                                double* Bop, int32_t* cexp) {
  const int64_t m = n - t0;
  const int ew = exp_above(__longlong_as_double((long long)*wmax));
  const double dn = pow2c(-ew), up = pow2c(ew);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    double mx = 0.0;
    for (int c = 0; c < nb; ++c) {
      const double v = V[t0 + i + c * ld], w = W[t0 + i + c * ld];
      Aop[i + c * m] = -v;
      Aop[i + (nb + c) * m] = -(w * dn);
      Bop[c + i * 2 * nb] = w;
      Bop[nb + c + i * 2 * nb] = v * up;
      mx = fmax(mx, fmax(fabs(w), fabs(v * up)));
    }
    cexp[i] = exp_above(mx);
  }
}

// Segment of the split update (and the list's end marker).
__global__ void k_trd_seg(GemmSeg* segs, int64_t m, int kk, const double* Aop, const double* Bop,
                          const int32_t* cexp, double* C, int64_t ldc, int S) {
  if (threadIdx.x != 0) return;
  const int64_t RT = (m + kSplitBM - 1) / kSplitBM, KB = (kk + kSplitBK - 1) / kSplitBK,
                CT = (m + kSplitBN - 1) / kSplitBN;
  GemmSeg sg;
  memset(&sg, 0, sizeof(sg));
  sg.A = Aop;
  sg.ars = 1;
  sg.lda = m;
  sg.rows = (int32_t)m;
  sg.kk = kk;
  sg.K = (int32_t)m;
  sg.Bd = Bop;
  sg.ldb = kk;
  sg.cexp = cexp;
  sg.C = C;
  sg.ldc = ldc;
  sg.acc = 1;
  sg.a_img = 0;
  sg.b_img = RT * KB * S * kSplitBM * kSplitBK;
  segs[0] = sg;
  GemmSeg end;
  memset(&end, 0, sizeof(end));
  end.it_a = RT * KB;
  end.it_b = CT * KB;
  end.it_t = RT * CT;
  end.a_img = sg.b_img + CT * KB * S * kSplitBN * kSplitBK;  // the images' end
  segs[1] = end;
}

// C (m x m) -= V W^T + W V^T in FP64 (V, W: m x nb, ld ldp), 32 x 32 tiles.
__global__ void __launch_bounds__(256) k_trd_syr2k_f64(int64_t m, int nb, const double* V, const double* W,
                                                      int64_t ldp, double* C, int64_t ldc) {
  __shared__ double sv[2][32][33], sw[2][32][33];
  const int64_t T = (m + 31) / 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int64_t b = blockIdx.x; b < T * T; b += gridDim.x) {
    const int64_t i0 = (b % T) * 32, j0 = (b / T) * 32;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int c0 = 0; c0 < nb; c0 += 32) {
      for (int r = ty; r < 32; r += 8) {
        const int c = c0 + tx;
        const bool okc = c < nb;
        sv[0][r][tx] = (okc && i0 + r < m) ? V[i0 + r + c * ldp] : 0.0;
        sw[0][r][tx] = (okc && i0 + r < m) ? W[i0 + r + c * ldp] : 0.0;
        sv[1][r][tx] = (okc && j0 + r < m) ? V[j0 + r + c * ldp] : 0.0;
        sw[1][r][tx] = (okc && j0 + r < m) ? W[j0 + r + c * ldp] : 0.0;
      }
      __syncthreads();
#pragma unroll 4
      for (int c = 0; c < 32; ++c) {
        const double vj = sv[1][tx][c], wj = sw[1][tx][c];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int r = ty + 8 * q;
          acc[q] = fma(sv[0][r][c], wj, fma(sw[0][r][c], vj, acc[q]));
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t i = i0 + ty + 8 * q, j = j0 + tx;
      if (i < m && j < m) C[i + j * ldc] -= acc[q];
    }
  }
}

// The last diagonal entries and off-diagonal once every reflector is applied.
__global__ void k_trd_tail(int64_t n, const double* A, int64_t lda, double* d, double* e, double* tau) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (n == 1) {
    d[0] = A[0];
    return;
  }
  d[n - 2] = A[(n - 2) + (n - 2) * lda];
  d[n - 1] = A[(n - 1) + (n - 1) * lda];
  e[n - 2] = A[(n - 1) + (n - 2) * lda];
  tau[n - 2] = 0.0;
}

// Range guard of the dense and band solvers (see launch_range_scale).
__global__ void __launch_bounds__(256) k_range_max(const double* A, int64_t rows, int64_t cols, int64_t ld, int lower,
                                                  unsigned long long* mx) {
  double m = 0.0;
  for (int64_t j = blockIdx.y; j < cols; j += gridDim.y)
    for (int64_t i = (lower ? j : 0) + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows;
         i += (int64_t)gridDim.x * blockDim.x) {
      const double x = A[i + j * ld];
      if (isfinite(x)) m = fmax(m, fabs(x));
    }
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) atomicMax(mx, (unsigned long long)__double_as_longlong(m));
}

__device__ __forceinline__ int range_exp(const unsigned long long* mx) {
  const double m = __longlong_as_double((long long)*mx);
  return (m > 0x1p400 || (m > 0.0 && m < 0x1p-400)) ? ilogb(m) : 0;
}

__global__ void __launch_bounds__(256) k_range_apply(double* A, int64_t rows, int64_t cols, int64_t ld, int lower,
                                                    const unsigned long long* mx, int* escale) {
  const int es = range_exp(mx);
  if (blockIdx.x == 0 && threadIdx.x == 0) *escale = es;
  if (es == 0) return;
  for (int64_t j = blockIdx.y; j < cols; j += gridDim.y)
    for (int64_t i = (lower ? j : 0) + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows;
         i += (int64_t)gridDim.x * blockDim.x)
      A[i + j * ld] = scale2(A[i + j * ld], -es);
}

__global__ void __launch_bounds__(256) k_range_unscale(double* x, int64_t n, const int* escale) {
  const int es = *escale;
  if (es == 0) return;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    x[t] = scale2(x[t], es);
}

cudaError_t launch_range_scale(double* A, int64_t rows, int64_t cols, int64_t ld, int lower, unsigned long long* mx,
                               int* escale, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(mx, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  // columns over grid.y, rows of a column over grid.x (coalesced, no index division)
  const dim3 g((unsigned)std::max<int64_t>(1, std::min<int64_t>((rows + 255) / 256, 8)),
               (unsigned)std::max<int64_t>(1, std::min<int64_t>(cols, 1216)));
  k_range_max<<<g, 256, 0, s>>>(A, rows, cols, ld, lower, mx);
  k_range_apply<<<g, 256, 0, s>>>(A, rows, cols, ld, lower, mx, escale);
  return cudaGetLastError();
}

cudaError_t launch_range_unscale(double* x, int64_t n, const int* escale, cudaStream_t s) {
  k_range_unscale<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096)), 256, 0, s>>>(x, n,
                                                                                                         escale);
  return cudaGetLastError();
}

int trd_panel_grid() {
  static int grid[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  if (!grid[dev]) {
    int sms = 0, per = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaFuncSetAttribute(k_trd_panel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(double) * kTrdSmemV)) != cudaSuccess)
      return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_trd_panel, kTrdThreads, sizeof(double) * kTrdSmemV) !=
            cudaSuccess ||
        per < 1)
      return 0;
    grid[dev] = std::min(sms, kTrdMaxBlocks);
  }
  return grid[dev];
}

cudaError_t launch_sym_fill(int64_t n, double* A, int64_t lda, cudaStream_t s) {
  const int64_t T = (n + 31) / 32;
  k_sym_fill<<<(unsigned)std::min<int64_t>(T * T, 4096), 256, 0, s>>>(n, A, lda);
  return cudaGetLastError();
}

size_t trd_panel_smem(int64_t n) { return n <= kTrdSmemV ? sizeof(double) * (size_t)std::max<int64_t>(n, 1) : 0; }

cudaError_t launch_trd_panel(const TrdPanel& P, int grid, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(P.bar, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  TrdPanel arg = P;
  arg.vsm = P.n <= kTrdSmemV ? 1 : 0;
  void* args[] = {&arg};
  return cudaLaunchCooperativeKernel((const void*)k_trd_panel, dim3(grid), dim3(kTrdThreads), args,
                                     trd_panel_smem(P.n), s);
}

cudaError_t launch_trd_update(const TrdUpdate& U, cudaStream_t s) {
  const int64_t m = U.n - U.t0;
  if (m <= 0 || U.nb <= 0) return cudaSuccess;
  double* C = U.A + U.t0 + U.t0 * U.lda;
  if (m < kTrdSplitMin) {
    const int64_t T = (m + 31) / 32;
    k_trd_syr2k_f64<<<(unsigned)std::min<int64_t>(T * T, 4096), 256, 0, s>>>(m, U.nb, U.V + U.t0, U.W + U.t0,
                                                                             U.ld, C, U.lda);
    return cudaGetLastError();
  }
  cudaError_t e = cudaMemsetAsync(U.wmax, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  k_trd_wmax<<<(unsigned)std::min<int64_t>((m * U.nb + 255) / 256, 1024), 256, 0, s>>>(U.t0, U.n, U.nb, U.W, U.ld,
                                                                                      U.wmax);
  k_trd_ops<<<(unsigned)std::min<int64_t>((m + 255) / 256, 1024), 256, 0, s>>>(U.t0, U.n, U.nb, U.V, U.W, U.ld,
                                                                               U.wmax, U.Aop, U.Bop, U.cexp);
  k_trd_seg<<<1, 32, 0, s>>>(U.segs, m, 2 * U.nb, U.Aop, U.Bop, U.cexp, C, U.lda, kTrdSlices);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_seg_split(U.segs, 1, kTrdSlices, U.status, U.budget, U.img, U.chunk_steps, s);
}

cudaError_t launch_trd_tail(int64_t n, const double* A, int64_t lda, double* d, double* e, double* tau,
                            cudaStream_t s) {
  k_trd_tail<<<1, 32, 0, s>>>(n, A, lda, d, e, tau);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Back-transform
// ---------------------------------------------------------------------------

// xexp[j]: 2^xexp[j] >= (1 + 2^-20) ||X(:, j)||, which bounds every entry of the column
// through the orthogonal updates (they keep its norm).
__global__ void __launch_bounds__(256) k_orm_xexp(int64_t rows, int64_t ncols, const double* X, int64_t ldx,
                                                 int32_t* xexp) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = w0; j < ncols; j += nw) {
    double s = 0.0;
    for (int64_t i = lane; i < rows; i += 32) s = fma(X[i + j * ldx], X[i + j * ldx], s);
    s = warp_sum(s);
    if (lane == 0) {
      const double nrm = sqrt(s) * (1.0 + 0x1p-20);
      int e = exp_above(nrm);
      if (pow2c(e) < nrm && e < 1022) ++e;
      xexp[j] = e;
    }
  }
}

// V_b (m_b x kbp, ld ldv): the reflectors b0 .. b0+kbp-1 over rows b0+1 .. n-1, explicit
// unit entry and zeros above it, from the lower triangle of the reduced A.
__global__ void __launch_bounds__(256) k_orm_v(int64_t n, int64_t b0, int kbp, const double* A, int64_t lda,
                                              double* Vb, int64_t ldv) {
  const int64_t mb = n - b0 - 1, total = mb * kbp;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % mb, c = t / mb;
    const int64_t r = b0 + 1 + i, k = b0 + c;
    Vb[i + c * ldv] = r < k + 1 ? 0.0 : (r == k + 1 ? 1.0 : A[r + k * lda]);
  }
}

// The split segments of one block of reflectors:
//   list 1 (2 ns segments): G_s = V_b(K_s, :)^T V_b(K_s, :) and Y_s = V_b(K_s, :)^T X(K_s, :)
//     over ns consecutive row ranges K_s of the block (partial sums, added by k_orm_z);
//   list 2 (1 segment): X(b0+1:n, :) += V_b Z.
__global__ void k_orm_segs(OrmStep O, GemmSeg* list1, GemmSeg* list2) {
  if (threadIdx.x != 0) return;
  const int S = O.S;
  const int64_t mb = O.mb, per = O.kper;
  int64_t ia = 0, ib = 0, it = 0, img = 0;
  for (int pass = 0; pass < 2; ++pass) {
    for (int s = 0; s < O.ns; ++s) {
      const int64_t k0 = s * per, kk = per < mb - k0 ? per : mb - k0;
      const int64_t K = pass == 0 ? O.kbp : O.ncols;
      const int64_t RT = (O.kbp + kSplitBM - 1) / kSplitBM, KB = (kk + kSplitBK - 1) / kSplitBK,
                    CT = (K + kSplitBN - 1) / kSplitBN;
      GemmSeg sg;
      memset(&sg, 0, sizeof(sg));
      sg.A = O.Vb + k0;  // A(r, c) = V_b(k0 + c, r)
      sg.ars = O.ldv;
      sg.lda = 1;
      sg.rows = O.kbp;
      sg.kk = (int32_t)kk;
      sg.K = (int32_t)K;
      if (pass == 0) {
        sg.Bd = O.Vb + k0;
        sg.ldb = O.ldv;
        sg.C = O.G + s * O.kbp * O.kbp;
        sg.ldc = O.kbp;
      } else {
        sg.Bd = O.X + O.b0 + 1 + k0;
        sg.ldb = O.ldx;
        sg.cexp = O.xexp;
        sg.C = O.Y + s * O.kbp * O.ncols;
        sg.ldc = O.kbp;
      }
      sg.it_a = ia;
      sg.it_b = ib;
      sg.it_t = it;
      sg.a_img = img;
      img += RT * KB * S * kSplitBM * kSplitBK;
      sg.b_img = img;
      img += CT * KB * S * kSplitBN * kSplitBK;
      ia += RT * KB;
      ib += CT * KB;
      it += RT * CT;
      list1[pass * O.ns + s] = sg;
    }
  }
  GemmSeg end;
  memset(&end, 0, sizeof(end));
  end.it_a = ia;
  end.it_b = ib;
  end.it_t = it;
  end.a_img = img;  // the images' end
  list1[2 * O.ns] = end;

  const int64_t RT = (mb + kSplitBM - 1) / kSplitBM, KB = (O.kbp + kSplitBK - 1) / kSplitBK,
                CT = (O.ncols + kSplitBN - 1) / kSplitBN;
  GemmSeg u;
  memset(&u, 0, sizeof(u));
  u.A = O.Vb;
  u.ars = 1;
  u.lda = O.ldv;
  u.rows = (int32_t)mb;
  u.kk = O.kbp;
  u.K = (int32_t)O.ncols;
  u.Bd = O.Z;
  u.ldb = O.kbp;
  u.cexp = O.zexp;
  u.C = O.X + O.b0 + 1;
  u.ldc = O.ldx;
  u.acc = 1;
  u.a_img = O.img2;
  u.b_img = O.img2 + RT * KB * S * kSplitBM * kSplitBK;
  list2[0] = u;
  GemmSeg e2;
  memset(&e2, 0, sizeof(e2));
  e2.it_a = RT * KB;
  e2.it_b = CT * KB;
  e2.it_t = RT * CT;
  e2.a_img = u.b_img + CT * KB * S * kSplitBN * kSplitBK;  // the images' end
  list2[1] = e2;
}

// Z = -T Y with T^-1 = diag(1/tau) + striu(G), G = sum_s G_s, Y = sum_s Y_s, by back
// substitution per column (a warp per column; lane t holds rows t, t+32, t+64, t+96);
// zexp[j] with |Z(:, j)| < 2^zexp[j].
__global__ void __launch_bounds__(kOrmZThreads, 1) k_orm_z(OrmStep O) {
  extern __shared__ double sG[];  // kbp x kbp (strict upper part used), then tau
  const int kbp = O.kbp;
  double* st = sG + kbp * kbp;
  for (int t = threadIdx.x; t < kbp * kbp; t += blockDim.x) {
    const int i = t % kbp, l = t / kbp;
    double s = 0.0;
    if (i < l)
      for (int q = 0; q < O.ns; ++q) s += O.G[q * kbp * kbp + t];
    sG[t] = s;
  }
  for (int t = threadIdx.x; t < kbp; t += blockDim.x) st[t] = O.tau[O.b0 + t];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = w0; j < O.ncols; j += nw) {
    double y[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = lane + 32 * q;
      double s = 0.0;
      if (i < kbp)
        for (int p = 0; p < O.ns; ++p) s += O.Y[(int64_t)p * kbp * O.ncols + i + j * kbp];
      y[q] = s;
    }
#pragma unroll
    for (int q = 3; q >= 0; --q) {
      for (int t = 31; t >= 0; --t) {
        const int l = 32 * q + t;
        if (l >= kbp) continue;
        const double zl = st[l] * __shfl_sync(0xffffffffu, y[q], t);
        if (lane == t) y[q] = zl;
#pragma unroll
        for (int qq = 0; qq <= q; ++qq) {
          const int i = lane + 32 * qq;
          if (i < l) y[qq] = fma(-sG[i + l * kbp], zl, y[qq]);
        }
      }
    }
    double mx = 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = lane + 32 * q;
      if (i < kbp) {
        O.Z[i + j * kbp] = -y[q];
        mx = fmax(mx, fabs(y[q]));
      }
    }
    mx = warp_max(mx);
    if (lane == 0) O.zexp[j] = exp_above(mx);
  }
}

cudaError_t launch_orm_xexp(int64_t rows, int64_t ncols, const double* X, int64_t ldx, int32_t* xexp,
                            cudaStream_t s) {
  k_orm_xexp<<<(unsigned)std::min<int64_t>((ncols * 32 + 255) / 256, 4096), 256, 0, s>>>(rows, ncols, X, ldx, xexp);
  return cudaGetLastError();
}

size_t orm_z_smem(int kbp) { return sizeof(double) * ((size_t)kbp * kbp + kbp); }

cudaError_t launch_orm_step(const OrmStep& O, const double* A, int64_t lda, cudaStream_t s) {
  const int64_t total = O.mb * O.kbp;
  k_orm_v<<<(unsigned)std::min<int64_t>((total + 255) / 256, 4096), 256, 0, s>>>(O.n, O.b0, O.kbp, A, lda, O.Vb,
                                                                                O.ldv);
  k_orm_segs<<<1, 32, 0, s>>>(O, O.list1, O.list2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_seg_split(O.list1, 2 * O.ns, O.S, O.status, O.budget, O.img, O.chunk_steps, s);
  if (e != cudaSuccess) return e;
  static bool attr[64] = {false};
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!attr[dev]) {
    e = cudaFuncSetAttribute(k_orm_z, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)orm_z_smem(kOrmKb));
    if (e != cudaSuccess) return e;
    attr[dev] = true;
  }
  const int64_t blocks = std::min<int64_t>((O.ncols + kOrmZThreads / 32 - 1) / (kOrmZThreads / 32), 1024);
  k_orm_z<<<(unsigned)blocks, kOrmZThreads, orm_z_smem(O.kbp), s>>>(O);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_seg_split(O.list2, 1, O.S, O.status, O.budget, O.img, O.chunk_steps, s);
}

}  // namespace tdc
