// tdc_banded.cu -- divide and conquer for symmetric band matrices (the band case Section 5
// points to), built from the merge's rank-one machinery.
//
// Tearing.  A node [lo, hi) of bandwidth b splits at m; its coupling block has rows
// r_k = m - b + k (k < b) with B_k(c) = A(m + c, r_k) (zero for c > k: outside the band).
// With s_k = sqrt(||B_k||), x_k = s_k e_{r_k}, y_k = B_k / s_k:
//   A = diag(A11 - sum_k x_k x_k^T, A22 - sum_k y_k y_k^T) + sum_k (x_k; y_k)(x_k; y_k)^T,
// i.e. A(r_k, r_k) -= ||B_k|| and the leading b x b corner of A22 -= sum_k B_k^T B_k / ||B_k||
// (b = 1 is Cuppen's tearing).  Rows with B_k = 0 give no term.
//
// Merge.  With the children's A1 = Q1 L1 Q1^T, A2 = Q2 L2 Q2^T and Q = diag(Q1, Q2), each
// term is one rank-one modification D + z z^T with z = Q^T (x_k; y_k), taken in turn: the
// poles sorted, deflated (type 1: rho |zhat_i| <= tol; type 2: a rotation when
// |t c s| <= tol for neighbouring poles, tol = 8 eps max(|D|max, |zhat|max), the tests of
// Section 3.2), the secular equation and the Cauchy-like update of the non-deflated
// columns (tdc_rank_one's kernels and the merge's product), the deflated columns copied.
#include "tdc_common.cuh"

namespace tdc {

namespace {
constexpr double kBdEps = 1.1102230246251565e-16;  // 2^-53
}  // namespace

// Tearing of the node split at m: the terms (s_k, y_k) into wv[k (b + 1) + 0..b] (s_k = 0:
// no term) and the corner updates of the band copy ABw (lower band storage, ld ldab).
__global__ void __launch_bounds__(256) k_bd_tear(double* ABw, int64_t ldab, int b, int64_t m, double* wv) {
  extern __shared__ double sb[];  // b x b: B_k(c) at sb[k * b + c], then b norms
  double* nrm = sb + b * b;
  for (int t = threadIdx.x; t < b * b; t += blockDim.x) {
    const int k = t / b, c = t % b;
    const int64_t r = m - b + k;
    sb[t] = c <= k ? ABw[(b - k + c) + r * ldab] : 0.0;  // A(m + c, r), m + c - r = b - k + c
  }
  __syncthreads();
  for (int k = threadIdx.x; k < b; k += blockDim.x) {
    double s2 = 0.0;
    for (int c = 0; c < b; ++c) s2 = fma(sb[k * b + c], sb[k * b + c], s2);
    const double nk = sqrt(s2);
    nrm[k] = nk;
    const double sk = sqrt(nk);
    wv[k * (b + 1)] = nk > 0.0 ? sk : 0.0;
    for (int c = 0; c < b; ++c) wv[k * (b + 1) + 1 + c] = nk > 0.0 ? sb[k * b + c] / sk : 0.0;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < b; k += blockDim.x) ABw[(m - b + k) * ldab] -= nrm[k];
  for (int t = threadIdx.x; t < b * b; t += blockDim.x) {
    const int c1 = t / b, c2 = t % b;
    if (c1 < c2) continue;
    double acc = 0.0;
    for (int k = 0; k < b; ++k)
      if (nrm[k] > 0.0) acc = fma(sb[k * b + c1], sb[k * b + c2] / nrm[k], acc);
    ABw[(c1 - c2) + (m + c2) * ldab] -= acc;
  }
}

// Lower triangle of the dense leaf block [lo, lo + L) (ld L) from the band copy.
__global__ void __launch_bounds__(256) k_bd_leaf_dense(const double* ABw, int64_t ldab, int b, int64_t lo, int64_t L,
                                                      double* Ad) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < L * L; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % L, j = t / L;
    if (i < j) continue;
    Ad[i + j * L] = (i - j <= b) ? ABw[(i - j) + (lo + j) * ldab] : 0.0;
  }
}

// z_j = s Q(ra, j) + sum_c y_c Q(rb + c, j), j < nn.
__global__ void __launch_bounds__(256) k_bd_z(int64_t nn, const double* Q, int64_t ldq, int64_t ra, int64_t rb, int b,
                                             const double* w, double* z) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nn; j += (int64_t)gridDim.x * blockDim.x) {
    const double* col = Q + j * ldq;
    double acc = w[0] * col[ra];
    for (int c = 0; c < b; ++c) acc = fma(w[1 + c], col[rb + c], acc);
    z[j] = acc;
  }
}

// (a, ia) before (b, ib) in a strict total order: ascending values, NaNs last, ties by
// index -- so that the ranks below always form a permutation.
__device__ __forceinline__ bool bd_before(double a, int64_t ia, double b, int64_t ib) {
  const bool na = a != a, nb = b != b;
  if (na || nb) return (!na && nb) || (na && nb && ia < ib);
  return a < b || (a == b && ia < ib);
}

// Stable rank sort: Ds[rank(i)] = D[i], zs likewise (z may be NULL), perm[rank(i)] = i.
__global__ void __launch_bounds__(256) k_bd_rank_sort(int64_t nn, const double* D, const double* z, double* Ds,
                                                     double* zs, int32_t* perm) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = D[i];
    int64_t rk = 0;
    for (int64_t j = 0; j < nn; ++j) rk += bd_before(D[j], j, v, i) ? 1 : 0;
    Ds[rk] = v;
    if (z) zs[rk] = z[i];
    perm[rk] = (int32_t)i;
  }
}

// Deflation scan over the sorted poles (one thread): zs normalised in place, kept / defl
// positions, rotations (pj, nj, c, s) on sorted positions, cnt = {K, nd, nrot}, *rho_out.
// A non-finite pole or weight records TDC_ENONFINITE and deflates every pole (no secular
// solve and no product run on it).
__global__ void k_bd_deflate(int64_t nn, double* Ds, double* zs, int32_t* kept, int32_t* defl, int32_t* rotp,
                             double* rotcs, int32_t* cnt, double* rho_out, int* status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s2 = 0.0;
  bool finite = true;
  for (int64_t i = 0; i < nn; ++i) {
    s2 = fma(zs[i], zs[i], s2);
    finite = finite && isfinite(zs[i]) && isfinite(Ds[i]);
  }
  if (!finite || !isfinite(s2)) {
    set_status(status, TDC_ENONFINITE);
    for (int64_t i = 0; i < nn; ++i) defl[i] = (int32_t)i;
    cnt[0] = 0;
    cnt[1] = (int32_t)nn;
    cnt[2] = 0;
    *rho_out = 0.0;
    return;
  }
  const double zn = sqrt(s2), rho = s2;
  double dmax = 0.0, zmax = 0.0;
  for (int64_t i = 0; i < nn; ++i) {
    if (zn > 0.0) zs[i] /= zn;
    dmax = fmax(dmax, fabs(Ds[i]));
    zmax = fmax(zmax, fabs(zs[i]));
  }
  const double tol = 8.0 * kBdEps * fmax(dmax, zmax);
  int32_t K = 0, nd = 0, nr = 0;
  int64_t pj = -1;
  for (int64_t j = 0; j < nn; ++j) {
    if (!(zn > 0.0) || rho * fabs(zs[j]) <= tol) {
      defl[nd++] = (int32_t)j;
      continue;
    }
    if (pj < 0) {
      pj = j;
      continue;
    }
    double s = zs[pj], c = zs[j];
    const double tau = hypot(c, s), t = Ds[j] - Ds[pj];
    c /= tau;
    s = -s / tau;
    if (fabs(t * c * s) <= tol) {
      zs[j] = tau;
      zs[pj] = 0.0;
      rotp[2 * nr] = (int32_t)pj;
      rotp[2 * nr + 1] = (int32_t)j;
      rotcs[2 * nr] = c;
      rotcs[2 * nr + 1] = s;
      ++nr;
      const double dp = Ds[pj], dn = Ds[j];
      Ds[pj] = dp * c * c + dn * s * s;
      Ds[j] = dp * s * s + dn * c * c;
      defl[nd++] = (int32_t)pj;
      pj = j;
    } else {
      kept[K++] = (int32_t)pj;
      pj = j;
    }
  }
  if (pj >= 0) kept[K++] = (int32_t)pj;
  cnt[0] = K;
  cnt[1] = nd;
  cnt[2] = nr;
  *rho_out = rho;
}

// The deflation rotations on the columns of Q (sorted position p is column perm[p]), in
// order, each row independently.
__global__ void __launch_bounds__(256) k_bd_rotate(int64_t nrows, double* Q, int64_t ldq, const int32_t* perm,
                                                  const int32_t* rotp, const double* rotcs, int nr, int* status) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nrows; r += (int64_t)gridDim.x * blockDim.x) {
    for (int t = 0; t < nr; ++t) {
      const int32_t pa = rotp[2 * t], pb = rotp[2 * t + 1];
      if (pa < 0 || pa >= nrows || pb < 0 || pb >= nrows || perm[pa] < 0 || perm[pa] >= nrows || perm[pb] < 0 ||
          perm[pb] >= nrows) {  // cannot happen for a permutation; never touch memory outside Q
        set_status(status, TDC_EUNSUPPORTED);
        continue;
      }
      double* a = Q + r + (int64_t)perm[pa] * ldq;
      double* bq = Q + r + (int64_t)perm[pb] * ldq;
      const double c = rotcs[2 * t], s = rotcs[2 * t + 1];
      const double x = *a, y = *bq;
      *a = c * x + s * y;
      *bq = c * y - s * x;
    }
  }
}

// Qw(:, t) = Q(:, perm[kept[t]]) for t < K, Q(:, perm[defl[t - K]]) after; the kept poles,
// their weights and the deflated values alongside.
__global__ void __launch_bounds__(256) k_bd_gather(int64_t nrows, const double* Q, int64_t ldq, const int32_t* perm,
                                                  const int32_t* kept, int K, const int32_t* defl, int nd,
                                                  const double* Ds, const double* zs, double* Qw, double* DK,
                                                  double* zK, double* Dd, int* status) {
  for (int64_t t = blockIdx.x; t < K + nd; t += gridDim.x) {
    const int32_t sp = t < K ? kept[t] : defl[t - K];
    if (t >= nrows || sp < 0 || sp >= nrows || perm[sp] < 0 || perm[sp] >= nrows) {  // cannot happen; never
      if (threadIdx.x == 0) set_status(status, TDC_EUNSUPPORTED);                   // read or write outside
      continue;
    }
    const double* src = Q + (int64_t)perm[sp] * ldq;
    double* dst = Qw + t * nrows;
    for (int64_t r = threadIdx.x; r < nrows; r += blockDim.x) dst[r] = src[r];
    if (threadIdx.x == 0) {
      if (t < K) {
        DK[t] = Ds[sp];
        zK[t] = zs[sp];
      } else {
        Dd[t - K] = Ds[sp];
      }
    }
  }
}

// Q(:, K + t) = Qw(:, K + t) (deflated columns); D = [roots; deflated values].
__global__ void __launch_bounds__(256) k_bd_finish(int64_t nrows, const double* Qw, double* Q, int64_t ldq, int K,
                                                  int nd, const double* DK, const int32_t* org, const double* tau,
                                                  const double* Dd, double* D) {
  for (int64_t t = blockIdx.x; t < K + nd && t < nrows; t += gridDim.x) {
    if (t >= K) {
      const double* src = Qw + t * nrows;
      double* dst = Q + t * ldq;
      for (int64_t r = threadIdx.x; r < nrows; r += blockDim.x) dst[r] = src[r];
    }
    if (threadIdx.x == 0) D[t] = t < K ? ((org[t] >= 0 && org[t] < K) ? DK[org[t]] + tau[t] : __longlong_as_double(0x7ff8000000000000ll)) : Dd[t - K];
  }
}

// Q(:, t) = Qw(:, t) for every column (the final order), lam = Ds.
__global__ void __launch_bounds__(256) k_bd_copy_back(int64_t nrows, int64_t ncols, const double* Qw, double* Q,
                                                     int64_t ldq) {
  for (int64_t t = blockIdx.x; t < ncols; t += gridDim.x) {
    const double* src = Qw + t * nrows;
    double* dst = Q + t * ldq;
    for (int64_t r = threadIdx.x; r < nrows; r += blockDim.x) dst[r] = src[r];
  }
}

__global__ void __launch_bounds__(256) k_bd_zero(int64_t rows, int64_t cols, double* Q, int64_t ldq) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < rows * cols;
       t += (int64_t)gridDim.x * blockDim.x)
    Q[t % rows + (t / rows) * ldq] = 0.0;
}

__global__ void __launch_bounds__(256) k_bd_copy_band(int64_t n, int b, const double* AB, int64_t ldab, double* ABw) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)(b + 1) * n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t % (b + 1), j = t / (b + 1);
    ABw[r + j * (b + 1)] = (j + r < n) ? AB[r + j * ldab] : 0.0;
  }
}

namespace {
unsigned grid_for(int64_t work, int64_t per = 256, int64_t cap = 4096) {
  const int64_t g = (work + per - 1) / per;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, cap));
}
}  // namespace

cudaError_t launch_bd_copy_band(int64_t n, int b, const double* AB, int64_t ldab, double* ABw, cudaStream_t s) {
  k_bd_copy_band<<<grid_for((int64_t)(b + 1) * n), 256, 0, s>>>(n, b, AB, ldab, ABw);
  return cudaGetLastError();
}
cudaError_t launch_bd_tear(double* ABw, int64_t ldab, int b, int64_t m, double* wv, cudaStream_t s) {
  if (b <= 0) return cudaSuccess;
  k_bd_tear<<<1, 256, sizeof(double) * (size_t)(b * b + b), s>>>(ABw, ldab, b, m, wv);
  return cudaGetLastError();
}
cudaError_t launch_bd_leaf_dense(const double* ABw, int64_t ldab, int b, int64_t lo, int64_t L, double* Ad,
                                 cudaStream_t s) {
  k_bd_leaf_dense<<<grid_for(L * L), 256, 0, s>>>(ABw, ldab, b, lo, L, Ad);
  return cudaGetLastError();
}
cudaError_t launch_bd_z(int64_t nn, const double* Q, int64_t ldq, int64_t ra, int64_t rb, int b, const double* w,
                        double* z, cudaStream_t s) {
  k_bd_z<<<grid_for(nn), 256, 0, s>>>(nn, Q, ldq, ra, rb, b, w, z);
  return cudaGetLastError();
}
cudaError_t launch_bd_sort(int64_t nn, const double* D, const double* z, double* Ds, double* zs, int32_t* perm,
                           cudaStream_t s) {
  k_bd_rank_sort<<<grid_for(nn), 256, 0, s>>>(nn, D, z, Ds, zs, perm);
  return cudaGetLastError();
}
cudaError_t launch_bd_deflate(int64_t nn, double* Ds, double* zs, int32_t* kept, int32_t* defl, int32_t* rotp,
                              double* rotcs, int32_t* cnt, double* rho, int* status, cudaStream_t s) {
  k_bd_deflate<<<1, 32, 0, s>>>(nn, Ds, zs, kept, defl, rotp, rotcs, cnt, rho, status);
  return cudaGetLastError();
}
cudaError_t launch_bd_rotate(int64_t nrows, double* Q, int64_t ldq, const int32_t* perm, const int32_t* rotp,
                             const double* rotcs, int nr, int* status, cudaStream_t s) {
  if (nr <= 0) return cudaSuccess;
  k_bd_rotate<<<grid_for(nrows), 256, 0, s>>>(nrows, Q, ldq, perm, rotp, rotcs, nr, status);
  return cudaGetLastError();
}
cudaError_t launch_bd_gather(int64_t nrows, const double* Q, int64_t ldq, const int32_t* perm, const int32_t* kept,
                             int K, const int32_t* defl, int nd, const double* Ds, const double* zs, double* Qw,
                             double* DK, double* zK, double* Dd, int* status, cudaStream_t s) {
  k_bd_gather<<<(unsigned)std::max(1, std::min(K + nd, 8192)), 256, 0, s>>>(nrows, Q, ldq, perm, kept, K, defl, nd, Ds,
                                                                            zs, Qw, DK, zK, Dd, status);
  return cudaGetLastError();
}
cudaError_t launch_bd_finish(int64_t nrows, const double* Qw, double* Q, int64_t ldq, int K, int nd, const double* DK,
                             const int32_t* org, const double* tau, const double* Dd, double* D, cudaStream_t s) {
  k_bd_finish<<<(unsigned)std::max(1, std::min(K + nd, 8192)), 256, 0, s>>>(nrows, Qw, Q, ldq, K, nd, DK, org, tau,
                                                                            Dd, D);
  return cudaGetLastError();
}
cudaError_t launch_bd_copy_back(int64_t nrows, int64_t ncols, const double* Qw, double* Q, int64_t ldq,
                                cudaStream_t s) {
  k_bd_copy_back<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ncols, 8192)), 256, 0, s>>>(nrows, ncols, Qw, Q,
                                                                                                 ldq);
  return cudaGetLastError();
}
cudaError_t launch_bd_zero(int64_t rows, int64_t cols, double* Q, int64_t ldq, cudaStream_t s) {
  k_bd_zero<<<grid_for(rows * cols), 256, 0, s>>>(rows, cols, Q, ldq);
  return cudaGetLastError();
}

}  // namespace tdc
