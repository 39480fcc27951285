// tdc_operands.cu -- products C = A B with a structured B given by generators (the
// further structured operands of Sections 1, 3.1 and 5: matrices of O(n) parameters):
// Toeplitz B(k, j) = t[k - j + n - 1], Hankel t[k + j], Vandermonde x_k^j, and the DFT
// matrix exp(-2 pi i k j / n) as its real and imaginary parts.  B is generated inside the
// product kernels -- the FP64 tiles of k_gemm_dense_seg and the digit images of k_split_b
// (struct_entry) -- so only the generators travel to the GPU (the point made in
// Section 5).  For the split product, column j of B enters scaled by 2^-eb_j with 2^eb_j
// above its largest |entry|: for Toeplitz / Hankel the maximum of |t| over the column's
// window of n consecutive generators, from a table of maxima over 2^L-wide windows
// (2^L <= n < 2^(L+1)) built in L doubling passes; for Vandermonde max|x|^j (with a
// margin for the rounding of the powers); for the DFT 0 (|entries| <= 1).  A enters
// scaled by 2^-eA from its largest row norm, and the product's column is scaled back by
// 2^eb_j (cexp) and 2^eA (oexp).
#include "tdc_common.cuh"

namespace tdc {

// One block: w0 = |t|, then L passes w_{l}[i] = max(w_{l-1}[i], w_{l-1}[i + 2^(l-1)]) between
// the two halves of `win` (2 x (2n - 1) doubles); eb[j] from the window of column j.
__global__ void __launch_bounds__(1024) k_tp_windows(int64_t n, const double* t, int kind, double* win,
                                                     int32_t* eb) {
  const int64_t len = 2 * n - 1;
  double* a = win;
  double* b = win + len;
  for (int64_t i = threadIdx.x; i < len; i += blockDim.x) a[i] = fabs(t[i]);
  __syncthreads();
  int64_t w = 1;
  while (2 * w <= n) {
    for (int64_t i = threadIdx.x; i + w < len; i += blockDim.x) b[i] = fmax(a[i], a[i + w]);
    __syncthreads();
    double* c = a;
    a = b;
    b = c;
    w *= 2;
  }
  // a holds maxima over windows of width w (w <= n < 2w)
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    const int64_t s = kind == 1 ? n - 1 - j : j;
    eb[j] = exp_above(fmax(a[s], a[s + n - w]));
  }
}

// Vandermonde: largest |x| (bits of a non-negative double in *mx, zero beforehand).
__global__ void __launch_bounds__(256) k_vd_max(int64_t n, const double* x, unsigned long long* mx) {
  double b = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b = fmax(b, fabs(x[i]));
  for (int off = 16; off > 0; off >>= 1) b = fmax(b, __shfl_xor_sync(0xffffffffu, b, off));
  if ((threadIdx.x & 31) == 0) atomicMax(mx, (unsigned long long)__double_as_longlong(b));
}

// eb_j from max|x|^j, raised by 2^-40 relative for the rounding of the computed powers
__global__ void __launch_bounds__(256) k_vd_exps(int64_t n, const unsigned long long* mx, int32_t* eb) {
  const double m = __longlong_as_double((long long)*mx);
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    eb[j] = exp_above(pow(m, (double)j) * (1.0 + 0x1p-40));
}

__global__ void __launch_bounds__(256) k_zero_i32(int64_t n, int32_t* a) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    a[j] = 0;
}

// cos(2 pi m / n) and -sin(2 pi m / n), m < n: the real and imaginary parts of the DFT
// matrix's entries exp(-2 pi i k j / n) at m = (k j) mod n.
__global__ void __launch_bounds__(256) k_dft_tables(int64_t n, double* cosv, double* msinv) {
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < n; m += (int64_t)gridDim.x * blockDim.x) {
    double sv, cv;
    sincospi(2.0 * ((double)m / (double)n), &sv, &cv);
    cosv[m] = cv;
    msinv[m] = -sv;
  }
}

// Largest squared row norm of A (m x n, lda) as the bits of a non-negative double.
__global__ void __launch_bounds__(256) k_tp_rows(int64_t m, int64_t n, const double* A, int64_t lda,
                                                unsigned long long* maxsq) {
  double best = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t k = 0; k < n; ++k) s = fma(A[i + k * lda], A[i + k * lda], s);
    best = fmax(best, s);
  }
  for (int off = 16; off > 0; off >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, off));
  if ((threadIdx.x & 31) == 0) atomicMax(maxsq, (unsigned long long)__double_as_longlong(best));
}

// eA with (largest row norm of A) 2^-eA < 1, and oexp[j] = eA: the product's columns are
// scaled back by 2^cexp[j] (B's column scale) and then by 2^oexp[j] (A's scale).
__global__ void __launch_bounds__(256) k_tp_exps(int64_t n, const unsigned long long* maxsq, int32_t* oexp,
                                                int32_t* eA) {
  const int e = exp_above(sqrt(__longlong_as_double((long long)*maxsq)));
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    oexp[j] = e;
  if (blockIdx.x == 0 && threadIdx.x == 0) *eA = e;
}

cudaError_t launch_operand_prep(int64_t m, int64_t n, const double* A, int64_t lda, const double* t, int kind,
                                double* winmax, int32_t* cexp, int32_t* oexp, int32_t* eA,
                                unsigned long long* maxsq, cudaStream_t s) {
  const unsigned g = (unsigned)std::min<int64_t>(1024, (n + 255) / 256);
  cudaError_t e = cudaSuccess;
  if (kind == 1 || kind == 2) {
    k_tp_windows<<<1, 1024, 0, s>>>(n, t, kind, winmax, cexp);
  } else if (kind == 3) {
    e = cudaMemsetAsync(maxsq, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    k_vd_max<<<g, 256, 0, s>>>(n, t, maxsq);
    k_vd_exps<<<g, 256, 0, s>>>(n, maxsq, cexp);
  } else {
    k_zero_i32<<<g, 256, 0, s>>>(n, cexp);
  }
  e = cudaMemsetAsync(maxsq, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  k_tp_rows<<<(unsigned)std::min<int64_t>(1024, (m + 255) / 256), 256, 0, s>>>(m, n, A, lda, maxsq);
  k_tp_exps<<<(unsigned)std::min<int64_t>(1024, (n + 255) / 256), 256, 0, s>>>(n, maxsq, oexp, eA);
  return cudaGetLastError();
}

cudaError_t launch_dft_tables(int64_t n, double* cosv, double* msinv, cudaStream_t s) {
  k_dft_tables<<<(unsigned)std::min<int64_t>(1024, (n + 255) / 256), 256, 0, s>>>(n, cosv, msinv);
  return cudaGetLastError();
}

}  // namespace tdc
