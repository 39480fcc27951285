// tdc_bdsdc.cu -- bidiagonal SVD through the divide-and-conquer eigensolver (the paper's
// introduction points to the divide and conquer for the bidiagonal SVD).  The upper
// bidiagonal B (d[n], e[n-1]) has the Golub-Kahan tridiagonal of order 2n with zero
// diagonal and off-diagonal (d_1, e_1, ..., e_{n-1}, d_n): its eigenvalues are
// +-sigma_i and the eigenvector of +sigma_i is (v_1, u_1, ..., v_n, u_n) / sqrt(2) with
// B v = sigma u, B^T u = sigma v.  The solver runs on that matrix; these kernels build
// it and read the singular triplets off the positive half (sigma descending).
#include "tdc_common.cuh"

namespace tdc {

__global__ void __launch_bounds__(256) k_gk_build(int64_t n, const double* d, const double* e, double* td,
                                                 double* te) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 2 * n; i += (int64_t)gridDim.x * blockDim.x) {
    td[i] = 0.0;
    if (i < 2 * n - 1) te[i] = (i & 1) ? e[i >> 1] : d[i >> 1];
  }
}

// sigma_i = lam[2n-1-i]; U(k, i) = sqrt(2) z_i(2k+1), VT(i, k) = sqrt(2) z_i(2k) with z_i the
// eigenvector of column 2n-1-i; 32 x 32 tiles of (i, k), VT through shared memory so that
// both outputs are written along their leading dimension.
__global__ void __launch_bounds__(256) k_gk_extract(int64_t n, const double* lam, const double* Q, int64_t ldq,
                                                   double* sigma, double* U, int64_t ldu, double* VT,
                                                   int64_t ldvt) {
  __shared__ double tv[32][33];
  const double r2 = 1.4142135623730951;  // sqrt(2) rounded to nearest
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t T = (n + 31) / 32;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    sigma[i] = lam[2 * n - 1 - i];
  for (int64_t b = blockIdx.x; b < T * T; b += gridDim.x) {
    const int64_t i0 = (b % T) * 32, k0 = (b / T) * 32;
    for (int r = ty; r < 32; r += 8) {
      const int64_t i = i0 + r, k = k0 + tx;
      if (i < n && k < n) {
        const double* z = Q + (2 * n - 1 - i) * ldq;
        U[k + i * ldu] = r2 * z[2 * k + 1];
        tv[r][tx] = r2 * z[2 * k];
      }
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
      const int64_t k = k0 + r, i = i0 + tx;
      if (i < n && k < n) VT[i + k * ldvt] = tv[tx][r];
    }
    __syncthreads();
  }
}

cudaError_t launch_gk_build(int64_t n, const double* d, const double* e, double* td, double* te, cudaStream_t s) {
  k_gk_build<<<(unsigned)std::min<int64_t>((2 * n + 255) / 256, 4096), 256, 0, s>>>(n, d, e, td, te);
  return cudaGetLastError();
}

cudaError_t launch_gk_extract(int64_t n, const double* lam, const double* Q, int64_t ldq, double* sigma, double* U,
                              int64_t ldu, double* VT, int64_t ldvt, cudaStream_t s) {
  const int64_t T = (n + 31) / 32;
  k_gk_extract<<<(unsigned)std::min<int64_t>(std::max<int64_t>(T * T, (n + 255) / 256), 8192), 256, 0, s>>>(
      n, lam, Q, ldq, sigma, U, ldu, VT, ldvt);
  return cudaGetLastError();
}

}  // namespace tdc
