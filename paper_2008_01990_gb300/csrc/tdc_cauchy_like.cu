// tdc_cauchy_like.cu -- the general Cauchy-like operand of Example 1 (Section 4):
// B_ij = u_i v_j / (d_i - w_j) with row nodes d, column nodes w and vectors u, v.
//
// B has the form of a merge's Qhat (Eq. (Q_Cauchy)): rows are poles d_i with weights
// u_i, and a column node is stored as an origin and an offset (Eq. (d-lambda)):
// org_j = the row node nearest to w_j, tau_j = w_j - d_org_j, so that every product
// kernel of the merge (dense, split, structured) generates B's entries from
// (d, org, tau, u, v) as it generates Qhat's.  The split products hold their operands
// as fixed-point digits of scale 1, so for them the operands are scaled by powers of
// two (exactly): A by 2^-eA with eA from its largest row norm, column j of B by
// 2^-eb_j with eb_j from its norm; then every row of A and column of B has norm <= 1,
// every entry of either and of the structured path's W = A B(:, T) is at most 1, and
// the product's column j is scaled back by 2^(eA + eb_j).
#include "tdc_common.cuh"

namespace tdc {

// org_j: the row node nearest to w_j (d ascending); tau_j = w_j - d[org_j].
__global__ void k_cl_nodes(int64_t n, const double* d, const double* w, int32_t* org, double* tau) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const double x = w[j];
    int64_t lo = 0, hi = n;  // first node >= x
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (d[mid] < x) lo = mid + 1; else hi = mid;
    }
    int64_t o = lo < n ? lo : n - 1;
    if (lo > 0 && (lo == n || x - d[lo - 1] <= d[lo] - x)) o = lo - 1;
    org[j] = (int32_t)o;
    tau[j] = x - d[o];
  }
}

// Column j (a warp): its norm |v_j| sqrt(sum_i (u_i / (d_i - w_j))^2), the exponent eb_j
// with norm 2^-eb_j < 1, and the column weight passed to the products: v_j 2^-eb_j
// (scale) or v_j.
__global__ void k_cl_cols(int64_t n, const double* d, const double* u, const double* v, const int32_t* org,
                          const double* tau, double* scol, int32_t* eb, int scale) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = warp; j < n; j += nwarps) {
    const double dorg = d[org[j]], tj = tau[j];
    double s = 0.0;
    for (int64_t i = lane; i < n; i += 32) {
      const double t = u[i] / ((d[i] - dorg) - tj);
      s = fma(t, t, s);
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) {
      const double nrm = fabs(v[j]) * sqrt(s);
      const int e = scale ? exp_above(nrm) : 0;
      eb[j] = e;
      scol[j] = scale ? v[j] * pow2c(-e) : v[j];
    }
  }
}

// The largest squared row norm of A (m x K, column-major, lda), as the bits of a
// non-negative double (ordered like the values) in *maxsq (zero beforehand).
__global__ void k_cl_rows(int64_t m, int64_t K, const double* A, int64_t lda, unsigned long long* maxsq) {
  double best = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t k = 0; k < K; ++k) {
      const double x = A[i + k * lda];
      s = fma(x, x, s);
    }
    best = fmax(best, s);
  }
  for (int off = 16; off > 0; off >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, off));
  if ((threadIdx.x & 31) == 0) atomicMax(maxsq, (unsigned long long)__double_as_longlong(best));
}

// eA with (largest row norm) 2^-eA < 1, and the product's column scales eA + eb_j.
__global__ void k_cl_exps(int64_t n, const unsigned long long* maxsq, const int32_t* eb, int32_t* cexp,
                          int32_t* eA) {
  const double mx = sqrt(__longlong_as_double((long long)*maxsq));
  const int e = exp_above(mx);
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    cexp[j] = eb[j] + e;
  if (blockIdx.x == 0 && threadIdx.x == 0) *eA = e;
}

// A segment written from the host learns A's scale.
__global__ void k_cl_patch(GemmSeg* seg, const int32_t* eA) {
  if (threadIdx.x == 0) seg->aexp = *eA;
}

cudaError_t launch_cauchy_like_prep(int64_t m, int64_t n, const double* A, int64_t lda, const double* d,
                                    const double* w, const double* u, const double* v, int32_t* org, double* tau,
                                    double* scol, int32_t* eb, int32_t* cexp, int32_t* eA,
                                    unsigned long long* maxsq, bool scale, cudaStream_t s) {
  const unsigned g1 = (unsigned)std::min<int64_t>(1024, (n + 255) / 256);
  k_cl_nodes<<<g1, 256, 0, s>>>(n, d, w, org, tau);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_cl_cols<<<(unsigned)std::min<int64_t>(4096, (n * 32 + 255) / 256), 256, 0, s>>>(n, d, u, v, org, tau, scol, eb,
                                                                                     scale ? 1 : 0);
  e = cudaGetLastError();
  if (e != cudaSuccess || !scale) return e;
  e = cudaMemsetAsync(maxsq, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  k_cl_rows<<<(unsigned)std::min<int64_t>(1024, (m + 255) / 256), 256, 0, s>>>(m, n, A, lda, maxsq);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_cl_exps<<<g1, 256, 0, s>>>(n, maxsq, eb, cexp, eA);
  return cudaGetLastError();
}

cudaError_t launch_cauchy_like_patch(GemmSeg* seg, const int32_t* eA, cudaStream_t s) {
  k_cl_patch<<<1, 32, 0, s>>>(seg, eA);
  return cudaGetLastError();
}

}  // namespace tdc
