// tdc_adjoint.cu -- reverse-mode derivative of the eigen-decomposition for the
// tridiagonal entries:
//     W = Q^T Q_bar,   M = diag(lam_bar) + F o skew(W),  F_ij = 1/(lam_j - lam_i),
//     R = Q M,         d_bar_i = <R_i,:, Q_i,:>,  e_bar_i = 2 <R_i,:, Q_i+1,:>
// (M symmetric, so Q M Q^T is symmetric and e_bar doubles its off-diagonal).
// Only the tridiagonal of Q M Q^T is formed; nothing of the merge tree is needed.
// Batched over problems of the same order stored back to back.
//
// The two n^3 products run on the split-precision tensor-core GEMM of the merge
// (base-256 BF16 digits, exact FP32 level sums, FP64 result): the left operand
// is Q^T or Q, whose rows have unit norm; the right operand (Q_bar or M, any
// magnitude) enters column by column scaled by a power of two that brings its
// largest entry below 1, and the product's column is scaled back exactly.
#include "tdc_common.cuh"

namespace tdc {

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

// cexp[b n + j]: exponent e of the largest |X_ij| of column j (= m 2^e, m in
// [0.5, 1)), clamped to [-1022, 1022]; magnitudes compared as integers.
__global__ void k_col_exp(int n, const double* X, int64_t ld, int64_t sX, int32_t* cexp) {
  const int b = blockIdx.y;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (w >= n) return;
  const int lane = threadIdx.x & 31;
  const unsigned long long* col = reinterpret_cast<const unsigned long long*>(X + b * sX + w * ld);
  unsigned long long mx = 0ull;
  for (int i = lane; i < n; i += 32) {
    const unsigned long long v = col[i] & 0x7fffffffffffffffull;
    if (v <= 0x7ff0000000000000ull && v > mx) mx = v;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ov = __shfl_xor_sync(0xffffffffu, mx, o);
    if (ov > mx) mx = ov;
  }
  if (lane == 0) {
    const int f = (int)(mx >> 52);
    int e = f == 0 ? -1022 : f - 1022;
    cexp[(int64_t)b * n + w] = e < -1022 ? -1022 : (e > 1022 ? 1022 : e);
  }
}

// Segment b of a batched product C_b = op(A_b) B_b (n x n each) for the split GEMM.
__global__ void k_adj_segs(int batch, int n, int S, const double* A, int64_t ars, int64_t lda, int64_t sA,
                           const double* B, int64_t ldb, int64_t sB, const int32_t* cexp, double* C, int64_t sC,
                           GemmSeg* segs) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b > batch) return;
  const int64_t RT = (n + kSplitBM - 1) / kSplitBM, KB = (n + kSplitBK - 1) / kSplitBK,
                CT = (n + kSplitBN - 1) / kSplitBN;
  const int64_t ta = RT * KB, tb = CT * KB, tt = RT * CT;
  const int64_t ael = ta * S * kSplitBM * kSplitBK, bel = tb * S * kSplitBN * kSplitBK;
  GemmSeg sg;
  memset(&sg, 0, sizeof(sg));
  sg.it_a = b * ta;
  sg.it_b = b * tb;
  sg.it_t = b * tt;
  sg.a_img = b * (ael + bel);
  sg.b_img = sg.a_img + ael;
  if (b < batch) {
    sg.A = A + b * sA;
    sg.ars = ars;
    sg.lda = lda;
    sg.rows = sg.kk = sg.K = n;
    sg.Bd = B + b * sB;
    sg.ldb = ldb;
    sg.cexp = cexp + (int64_t)b * n;
    sg.C = C + b * sC;
    sg.ldc = n;
  }
  segs[b] = sg;
}

int64_t adjoint_split_img_elems(int batch, int64_t n) {
  const int64_t RT = (n + kSplitBM - 1) / kSplitBM, KB = (n + kSplitBK - 1) / kSplitBK,
                CT = (n + kSplitBN - 1) / kSplitBN;
  return (int64_t)batch * (RT * KB * kAdjSlices * kSplitBM * kSplitBK + CT * KB * kAdjSlices * kSplitBN * kSplitBK);
}

// ws: W, R (batch n^2 doubles each), then the column exponents (batch n int32),
// the segments (batch + 1) and the digit images (adjoint_split_img_elems).
cudaError_t launch_adjoint(int batch, int n, const double* lam, const double* Q, int64_t ldq, int64_t sQ,
                           const double* lam_bar, const double* Q_bar, int64_t sQb, double* d_bar,
                           double* e_bar, double* ws, int* status, long long spin_budget, cudaStream_t s) {
  if (batch <= 0 || n <= 0) return cudaSuccess;
  const int64_t nn = (int64_t)n * n;
  double* W = ws;                // batch x n x n
  double* R = ws + batch * nn;   // batch x n x n
  int32_t* cexp = reinterpret_cast<int32_t*>(R + batch * nn);
  uintptr_t sp = reinterpret_cast<uintptr_t>(cexp + (int64_t)batch * n);
  sp = (sp + 255) & ~(uintptr_t)255;
  GemmSeg* segs = reinterpret_cast<GemmSeg*>(sp);
  sp = reinterpret_cast<uintptr_t>(segs + batch + 1);
  sp = (sp + 255) & ~(uintptr_t)255;
  __nv_bfloat16* img = reinterpret_cast<__nv_bfloat16*>(sp);
  const dim3 cg((unsigned)((n * 32 + 255) / 256), batch);
  const unsigned sgrid = (unsigned)((batch + 1 + 127) / 128);
  cudaError_t e;
  if (Q_bar) {
    // W = Q^T Q_bar: A(i, k) = Q(k, i)
    k_col_exp<<<cg, 256, 0, s>>>(n, Q_bar, ldq, sQb, cexp);
    k_adj_segs<<<sgrid, 128, 0, s>>>(batch, n, kAdjSlices, Q, ldq, 1, sQ, Q_bar, ldq, sQb, cexp, W, nn, segs);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_seg_split(segs, batch, kAdjSlices, status, spin_budget, img, 0, s);
    if (e != cudaSuccess) return e;
  } else {
    e = cudaMemsetAsync(W, 0, sizeof(double) * batch * nn, s);
    if (e != cudaSuccess) return e;
  }
  const unsigned mb = (unsigned)std::min<int64_t>((nn + 255) / 256, 1024);
  k_adj_m<<<dim3(mb, batch), 256, 0, s>>>(n, W, nn, lam, n, lam_bar, Q_bar != nullptr);
  // R = Q M: A(i, k) = Q(i, k)
  k_col_exp<<<cg, 256, 0, s>>>(n, W, n, nn, cexp);
  k_adj_segs<<<sgrid, 128, 0, s>>>(batch, n, kAdjSlices, Q, 1, ldq, sQ, W, n, nn, cexp, R, nn, segs);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_seg_split(segs, batch, kAdjSlices, status, spin_budget, img, 0, s);
  if (e != cudaSuccess) return e;
  k_adj_dots<<<dim3((unsigned)((n * 32 + 255) / 256), batch), 256, 0, s>>>(n, R, nn, Q, ldq, sQ, d_bar, n, e_bar,
                                                                          n > 1 ? n - 1 : 1);
  return cudaGetLastError();
}

}  // namespace tdc
