// tdc_adjoint.cu -- reverse-mode derivative of the eigen-decomposition for the
// tridiagonal entries:
//     W = Q^T Q_bar,   M = diag(lam_bar) + F o skew(W),  F_ij = 1/(lam_j - lam_i),
//     R = Q M,         d_bar_i = <R_i,:, Q_i,:>,  e_bar_i = 2 <R_i,:, Q_i+1,:>
// (M symmetric, so Q M Q^T is symmetric and e_bar doubles its off-diagonal).
// Only the tridiagonal of Q M Q^T is formed; nothing of the merge tree is needed.
// Batched over problems of the same order stored back to back.
#include "tdc_common.cuh"

namespace tdc {

namespace {
constexpr int BM = 128, BN = 64, BK = 16, kThreads = 256;
}

// C[b] = op(A[b]) * B[b] for square n x n FP64 matrices (column-major), op = A^T
// when TA.  128 x 64 tiles, 256 threads with 8 x 4 outputs each.
template <bool TA>
__global__ void __launch_bounds__(kThreads, 2) k_gemm64(int n, const double* A, int64_t lda, int64_t sA,
                                                        const double* B, int64_t ldb, int64_t sB, double* C,
                                                        int64_t ldc, int64_t sC) {
  __shared__ double As[BK][BM];
  __shared__ double Bs[BK][BN];
  const int b = blockIdx.z;
  A += b * sA;
  B += b * sB;
  C += b * sC;
  const int r0 = blockIdx.x * BM, c0 = blockIdx.y * BN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[i][c] = 0.0;
  for (int k0 = 0; k0 < n; k0 += BK) {
    __syncthreads();
#pragma unroll
    for (int e = 0; e < (BK * BM) / kThreads; ++e) {
      const int idx = tid + e * kThreads;
      int k, r;
      if (TA) { k = idx % BK; r = idx / BK; }  // A^T(r, k) = A(k, r): k contiguous
      else { r = idx % BM; k = idx / BM; }
      const int row = r0 + r, kk = k0 + k;
      double x = 0.0;
      if (row < n && kk < n) x = TA ? A[kk + (int64_t)row * lda] : A[row + (int64_t)kk * lda];
      As[k][r] = x;
    }
#pragma unroll
    for (int e = 0; e < (BK * BN) / kThreads; ++e) {
      const int idx = tid + e * kThreads;
      const int k = idx % BK, c = idx / BK;
      const int kk = k0 + k, col = c0 + c;
      Bs[k][c] = (kk < n && col < n) ? B[kk + (int64_t)col * ldb] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
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
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int col = c0 + tx * 4 + c;
    if (col >= n) continue;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int row = r0 + ty * 8 + i;
      if (row < n) C[row + (int64_t)col * ldc] = acc[i][c];
    }
  }
}

// M = diag(lam_bar) + F o skew(W), in place over W (each thread owns a pair (i,j), (j,i)).
__global__ void k_adj_m(int n, double* W, int64_t sW, const double* lam, int64_t sL, const double* lam_bar,
                        bool have_qbar) {
  const int b = blockIdx.y;
  double* w = W + b * sW;
  const double* l = lam + b * sL;
  const double* lb = lam_bar ? lam_bar + b * sL : nullptr;
  const int64_t total = (int64_t)n * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), j = (int)(t / n);
    if (i > j) continue;
    if (i == j) {
      w[i + (int64_t)i * n] = lb ? lb[i] : 0.0;
      continue;
    }
    double mij = 0.0;
    if (have_qbar) {
      const double sk = 0.5 * (w[i + (int64_t)j * n] - w[j + (int64_t)i * n]);
      mij = sk / (l[j] - l[i]);  // F_ij skew_ij; the (j, i) entry is F_ji skew_ji = the same
    }
    w[i + (int64_t)j * n] = mij;
    w[j + (int64_t)i * n] = mij;
  }
}

// d_bar_i = <R_i, Q_i>, e_bar_i = 2 <R_i, Q_{i+1}>; one warp per row.
__global__ void k_adj_dots(int n, const double* R, int64_t sR, const double* Q, int64_t ldq, int64_t sQ,
                           double* d_bar, int64_t sd, double* e_bar, int64_t se) {
  const int b = blockIdx.y;
  const int64_t wrow = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (wrow >= n) return;
  const int i = (int)wrow, lane = threadIdx.x & 31;
  const double* r = R + b * sR;
  const double* q = Q + b * sQ;
  double sd0 = 0.0, se0 = 0.0;
  for (int k = lane; k < n; k += 32) {
    const double rik = r[i + (int64_t)k * n];
    sd0 = fma(rik, q[i + (int64_t)k * ldq], sd0);
    if (i + 1 < n) se0 = fma(rik, q[i + 1 + (int64_t)k * ldq], se0);
  }
  sd0 = warp_sum(sd0);
  se0 = warp_sum(se0);
  if (lane == 0) {
    d_bar[b * sd + i] = sd0;
    if (i + 1 < n) e_bar[b * se + i] = 2.0 * se0;
  }
}

cudaError_t launch_adjoint(int batch, int n, const double* lam, const double* Q, int64_t ldq, int64_t sQ,
                           const double* lam_bar, const double* Q_bar, int64_t sQb, double* d_bar,
                           double* e_bar, double* ws, cudaStream_t s) {
  if (batch <= 0 || n <= 0) return cudaSuccess;
  const int64_t nn = (int64_t)n * n;
  double* W = ws;                // batch x n x n
  double* R = ws + batch * nn;   // batch x n x n
  const dim3 grid((n + BM - 1) / BM, (n + BN - 1) / BN, batch);
  if (Q_bar) {
    k_gemm64<true><<<grid, kThreads, 0, s>>>(n, Q, ldq, sQ, Q_bar, ldq, sQb, W, n, nn);
  } else {
    cudaError_t e = cudaMemsetAsync(W, 0, sizeof(double) * batch * nn, s);
    if (e != cudaSuccess) return e;
  }
  const unsigned mb = (unsigned)std::min<int64_t>((nn + 255) / 256, 1024);
  k_adj_m<<<dim3(mb, batch), 256, 0, s>>>(n, W, nn, lam, n, lam_bar, Q_bar != nullptr);
  k_gemm64<false><<<grid, kThreads, 0, s>>>(n, Q, ldq, sQ, W, n, nn, R, n, nn);
  k_adj_dots<<<dim3((unsigned)((n * 32 + 255) / 256), batch), 256, 0, s>>>(n, R, nn, Q, ldq, sQ, d_bar, n, e_bar,
                                                                          n > 1 ? n - 1 : 1);
  return cudaGetLastError();
}

}  // namespace tdc
