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

__device__ __forceinline__ double pow2i(int e) { return __hiloint2double((1023 + e) << 20, 0); }

// exponent e with |x| < 2^e for the largest magnitude x (0 for x = 0)
__device__ __forceinline__ int exp_above(double mx) { return mx > 0.0 ? ilogb(mx) + 1 : 0; }

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier of a cooperative launch: a growing arrival counter (zero before the
// launch); a block's b-th barrier waits until b * gridDim.x arrivals.  The wait gives up
// after `budget` polls, records TDC_ETIMEOUT and returns false in the whole block.
__device__ bool grid_barrier(unsigned* ctr, unsigned& target, long long budget, int* status, int* s_flag) {
  __syncthreads();
  target += gridDim.x;
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(ctr, 1u);
    int ok = 1;
    long long it = 0;
    while (ld_acquire_u32(ctr) < target) {
      if (++it > budget) {
        ok = 0;
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
    if (!ok) set_status(status, TDC_ETIMEOUT);
    *s_flag = ok;
  }
  __syncthreads();
  return *s_flag != 0;
}

// gamma = w~^T v = tau (v^T y - 2 pw^T pv) of a column with c earlier panel columns, from
// the per-block partials of v^T y (one warp, the same order in every block)
__device__ __forceinline__ double gamma_of(const double* pvy, const double* pw, const double* pv, int c, double tc) {
  const int lane = threadIdx.x & 31;
  double s = 0.0, q = 0.0;
  for (int b = lane; b < (int)gridDim.x; b += 32) s += pvy[b];
  for (int i = lane; i < c; i += 32) q = fma(pw[i], pv[i], q);
  s = warp_sum(s);
  q = warp_sum(q);
  return tc * (s - 2.0 * q);
}

// sum over a block's warps in warp order (thread 0 gets the result)
__device__ __forceinline__ double block_sum_ordered(double v, double* s_red) {
  v = warp_sum(v);
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

__global__ void __launch_bounds__(kTrdThreads, 1) k_trd_panel(TrdPanel P) {
  __shared__ double s_vk[kTrdNb], s_wk[kTrdNb], s_pw[kTrdNb], s_pv[kTrdNb];
  __shared__ double s_red[kTrdThreads / 32];
  __shared__ double s_scal[4];
  __shared__ int s_flag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t n = P.n, ld = P.n;
  const int64_t G = (int64_t)gridDim.x * blockDim.x, g = (int64_t)blockIdx.x * blockDim.x + tid;
  const int64_t GW = G >> 5, gw = g >> 5;
  unsigned target = 0;
  double* __restrict__ A = P.A;
  double* __restrict__ V = P.V;
  double* __restrict__ W = P.W;
  const int64_t lda = P.lda;

  for (int j = 0; j < P.nbp; ++j) {
    const int64_t k = P.p + j;
    // ---- (1) finish w of column j-1, update column k with the panel so far
    double tprev = 0.0, gam = 0.0;
    if (j > 0) {
      tprev = P.tau[k - 1];
      for (int c = tid; c < j - 1; c += blockDim.x) {
        s_pw[c] = P.pw[c];
        s_pv[c] = P.pv[c];
        s_vk[c] = V[k + c * ld];
        s_wk[c] = W[k + c * ld];
      }
      if (tid == 0) s_vk[j - 1] = V[k + (j - 1) * ld];
      __syncthreads();
      if (warp == 0) {
        const double gm = gamma_of(P.pvy, s_pw, s_pv, j - 1, tprev);
        double f = 0.0;
        for (int c = lane; c < j - 1; c += 32) f = fma(s_vk[c], s_pw[c], fma(s_wk[c], s_pv[c], f));
        f = warp_sum(f);
        if (lane == 0) {
          s_scal[0] = gm;
          s_wk[j - 1] = tprev * (P.y[k] - f) - 0.5 * tprev * gm * s_vk[j - 1];
        }
      }
      __syncthreads();
      gam = s_scal[0];
    }
    double ss = 0.0;
    for (int64_t r = k + g; r < n; r += G) {
      double a = A[r + k * lda];
      if (j > 0) {
        double f = 0.0, u = 0.0;
        for (int c = 0; c < j - 1; ++c) {
          const double vrc = V[r + c * ld], wrc = W[r + c * ld];
          f = fma(vrc, s_pw[c], fma(wrc, s_pv[c], f));
          u = fma(vrc, s_wk[c], fma(wrc, s_vk[c], u));
        }
        const double vr = V[r + (j - 1) * ld];
        const double wr = (r == k) ? s_wk[j - 1] : tprev * (P.y[r] - f) - 0.5 * tprev * gam * vr;
        W[r + (j - 1) * ld] = wr;
        u = fma(vr, s_wk[j - 1], fma(wr, s_vk[j - 1], u));
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
    {
      const double t = block_sum_ordered(ss, s_red);
      if (tid == 0) P.ps[blockIdx.x] = t;
    }
    if (!grid_barrier(P.bar, target, P.budget, P.status, &s_flag)) return;

    // ---- (2) the reflector of column k; A22 v and the panel dots
    if (warp == 0) {
      double s = 0.0;
      for (int b = lane; b < (int)gridDim.x; b += 32) s += P.ps[b];
      s = warp_sum(s);
      if (lane == 0) {
        const double alpha = P.x[k + 1];
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
      const double v = r <= k ? 0.0 : (r == k + 1 ? 1.0 : P.x[r] * sc);
      V[r + j * ld] = v;
      if (r >= k + 2) A[r + k * lda] = v;
    }
    const int64_t ncol = n - k - 1, items = ncol + 2 * (int64_t)j;
    double vy = 0.0;
    for (int64_t t = gw; t < items; t += GW) {
      const double* col;
      if (t < ncol) col = A + (k + 1 + t) * lda;
      else col = (((t - ncol) & 1) ? V : W) + ((t - ncol) >> 1) * ld;
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      int64_t r = k + 1 + lane;
      if (r == k + 1) {  // lane 0's first row: v = 1
        a0 = col[r];
        r += 32;
      } else if (r < n) {
        a0 = col[r] * (P.x[r] * sc);
        r += 32;
      }
      for (; r + 96 < n; r += 128) {
        a0 = fma(col[r], P.x[r] * sc, a0);
        a1 = fma(col[r + 32], P.x[r + 32] * sc, a1);
        a2 = fma(col[r + 64], P.x[r + 64] * sc, a2);
        a3 = fma(col[r + 96], P.x[r + 96] * sc, a3);
      }
      for (; r < n; r += 32) a0 = fma(col[r], P.x[r] * sc, a0);
      const double dot = warp_sum((a0 + a1) + (a2 + a3));
      if (lane == 0) {
        if (t < ncol) {
          const int64_t c = k + 1 + t;
          P.y[c] = dot;
          vy = fma(c == k + 1 ? 1.0 : P.x[c] * sc, dot, vy);
        } else if ((t - ncol) & 1) {
          P.pv[(t - ncol) >> 1] = dot;
        } else {
          P.pw[(t - ncol) >> 1] = dot;
        }
      }
    }
    {
      const double t = block_sum_ordered(vy, s_red);
      if (tid == 0) P.pvy[blockIdx.x] = t;
    }
    if (!grid_barrier(P.bar, target, P.budget, P.status, &s_flag)) return;
  }

  // ---- w of the panel's last column on the trailing rows
  const int jl = P.nbp - 1;
  const double tl = P.tau[P.p + jl];
  for (int c = tid; c < jl; c += blockDim.x) {
    s_pw[c] = P.pw[c];
    s_pv[c] = P.pv[c];
  }
  __syncthreads();
  if (warp == 0) {
    const double gm = gamma_of(P.pvy, s_pw, s_pv, jl, tl);
    if (lane == 0) s_scal[0] = gm;
  }
  __syncthreads();
  const double gam = s_scal[0];
  for (int64_t r = P.p + P.nbp + g; r < n; r += G) {
    double f = 0.0;
    for (int c = 0; c < jl; ++c) f = fma(V[r + c * ld], s_pw[c], fma(W[r + c * ld], s_pv[c], f));
    W[r + jl * ld] = tl * (P.y[r] - f) - 0.5 * tl * gam * V[r + jl * ld];
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
  const double dn = pow2i(-ew), up = pow2i(ew);
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

int trd_panel_grid() {
  static int grid[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  if (!grid[dev]) {
    int sms = 0, per = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_trd_panel, kTrdThreads, 0) != cudaSuccess || per < 1)
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

cudaError_t launch_trd_panel(const TrdPanel& P, int grid, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(P.bar, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  TrdPanel arg = P;
  void* args[] = {&arg};
  return cudaLaunchCooperativeKernel((const void*)k_trd_panel, dim3(grid), dim3(kTrdThreads), args, 0, s);
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
      if (pow2i(e) < nrm) ++e;
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
