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

// Leaves, one block each.  k_bd_leaf_trd: the dense symmetric block of the torn band
// (both triangles) reduced to tridiagonal form by Householder reflectors, column by column
// (the reduction of the dense solver, unblocked: a leaf has at most 8b or 128 rows and the
// block stays in L2): for column k, x = A(k+1:L, k), alpha = x_0, sigma = ||x(1:)||,
// beta = -sign(alpha) hypot(alpha, sigma), tau = (beta - alpha) / beta,
// v = [1, x(1:) / (alpha - beta)] (stored below the subdiagonal), p = tau A22 v,
// w = p - (tau / 2)(p^T v) v, A22 -= v w^T + w v^T (sigma = 0: tau = 0, nothing applied).
__device__ __forceinline__ double bd_block_sum(double v, double* red) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  return t;
}

__global__ void __launch_bounds__(kBdLeafThreads) k_bd_leaf_trd(BdLeafArgs P, BdLeafTable T) {
  __shared__ double v[512], pw[512], red[32];
  __shared__ double s_tau, s_scal;
  __shared__ int s_skip;
  const int64_t lo = T.lo[blockIdx.x];
  const int L = T.L[blockIdx.x];
  if (L <= 0 || L > 512) return;
  double* A = P.Ab + lo * P.lmax;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  for (int t = tid; t < L * L; t += blockDim.x) {
    const int i = t % L, j = t / L;
    const int r = i > j ? i - j : j - i, c = i > j ? j : i;
    A[t] = r <= P.b ? P.ABw[r + (lo + c) * P.ldab] : 0.0;
  }
  __syncthreads();
  for (int k = 0; k + 2 < L; ++k) {
    const int m = L - k - 1;
    double* x = A + (k + 1) + (int64_t)k * L;
    double* A22 = A + (k + 1) + (int64_t)(k + 1) * L;
    double ss = 0.0;
    for (int i = tid; i < m; i += blockDim.x) {
      const double xi = x[i];
      v[i] = xi;
      if (i > 0) ss = fma(xi, xi, ss);
    }
    ss = bd_block_sum(ss, red);
    if (tid == 0) {
      const double alpha = v[0];
      P.d[lo + k] = A[k + (int64_t)k * L];
      if (ss == 0.0) {
        s_skip = 1;
        P.e[lo + k] = alpha;
        P.tau[lo + k] = 0.0;
      } else {
        const double beta = -copysign(hypot(alpha, sqrt(ss)), alpha);
        s_skip = 0;
        s_tau = (beta - alpha) / beta;
        s_scal = 1.0 / (alpha - beta);
        P.e[lo + k] = beta;
        P.tau[lo + k] = s_tau;
      }
    }
    __syncthreads();
    if (s_skip) continue;
    const double tau = s_tau, scal = s_scal;
    for (int i = tid; i < m; i += blockDim.x) {
      const double vi = i == 0 ? 1.0 : v[i] * scal;
      v[i] = vi;
      if (i > 0) x[i] = vi;
    }
    __syncthreads();
    // p_i = tau (A22 v)_i: column i of the symmetric A22 against v, a warp per column
    for (int i = wid; i < m; i += nw) {
      const double* col = A22 + (int64_t)i * L;
      double acc = 0.0;
      for (int j = lane; j < m; j += 32) acc = fma(col[j], v[j], acc);
      acc = warp_sum(acc);
      if (lane == 0) pw[i] = tau * acc;
    }
    __syncthreads();
    double pv = 0.0;
    for (int i = tid; i < m; i += blockDim.x) pv = fma(pw[i], v[i], pv);
    pv = bd_block_sum(pv, red);
    const double h = 0.5 * tau * pv;
    for (int i = tid; i < m; i += blockDim.x) pw[i] = fma(-h, v[i], pw[i]);
    __syncthreads();
    for (int t = tid; t < m * m; t += blockDim.x) {
      const int i = t % m, j = t / m;
      // the same two products and one addition for (i, j) and (j, i): A22 stays symmetric
      A22[i + (int64_t)j * L] -= __dadd_rn(__dmul_rn(v[i], pw[j]), __dmul_rn(pw[i], v[j]));
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (L == 1) {
      P.d[lo] = A[0];
    } else {
      P.d[lo + L - 2] = A[(L - 2) + (int64_t)(L - 2) * L];
      P.d[lo + L - 1] = A[(L - 1) + (int64_t)(L - 1) * L];
      P.e[lo + L - 2] = A[(L - 1) + (int64_t)(L - 2) * L];
      P.tau[lo + L - 2] = 0.0;
    }
  }
}

// k_bd_leaf_back: Q(lo:lo+L, lo:lo+L) = H_0 ... H_{L-3} Z, Z the leaf tridiagonal's
// eigenvectors (Zb, ld L): Z copied into Q's block, then the reflectors applied last
// first, each as y = v^T Z(k+1:L, :) (a warp per column) and Z(k+1:L, :) -= tau v y.
__global__ void __launch_bounds__(kBdLeafThreads) k_bd_leaf_back(BdLeafArgs P, BdLeafTable T) {
  __shared__ double v[512], y[512];
  const int64_t lo = T.lo[blockIdx.x];
  const int L = T.L[blockIdx.x];
  if (L <= 0 || L > 512) return;
  const double* A = P.Ab + lo * P.lmax;
  const double* Z = P.Zb + lo * P.lmax;
  double* Qb = P.Q + lo + lo * P.ldq;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  for (int t = tid; t < L * L; t += blockDim.x) {
    const int i = t % L, j = t / L;
    Qb[i + (int64_t)j * P.ldq] = Z[t];
  }
  __syncthreads();
  for (int k = L - 3; k >= 0; --k) {
    const double tau = P.tau[lo + k];
    if (tau == 0.0) continue;  // uniform across the block
    const int m = L - k - 1;
    for (int i = tid; i < m; i += blockDim.x) v[i] = i == 0 ? 1.0 : A[(k + 1 + i) + (int64_t)k * L];
    __syncthreads();
    for (int j = wid; j < L; j += nw) {
      const double* col = Qb + (k + 1) + (int64_t)j * P.ldq;
      double acc = 0.0;
      for (int i = lane; i < m; i += 32) acc = fma(v[i], col[i], acc);
      acc = warp_sum(acc);
      if (lane == 0) y[j] = tau * acc;
    }
    __syncthreads();
    for (int t = tid; t < m * L; t += blockDim.x) {
      const int i = t % m, j = t / m;
      Qb[(k + 1 + i) + (int64_t)j * P.ldq] -= v[i] * y[j];
    }
    __syncthreads();
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

// Stable sort by rank in two kernels.  k_bd_chunk_sort: one block per chunk of ch entries
// (ch = kBdChunk, or the power of two at or above nn when that is smaller) sorts (D[i], i)
// by bd_before with a bitonic network in shared memory (entries past nn pad the chunk and
// sort last), writing the chunk's sorted keys and indices.
// k_bd_rank: entry i at sorted place p of its chunk has rank p + the count of entries before
// it in every other chunk (a binary search each); Ds[rank] = D[i], zs likewise (z may be
// NULL), perm[rank] = i.  The ranks are those of the total order, a permutation.
constexpr int kBdChunk = 2048;

__device__ __forceinline__ bool bd_before_pad(double a, int64_t ia, double b, int64_t ib, int64_t nn) {
  if (ia >= nn || ib >= nn) return ia < nn || (ib >= nn && ia < ib);
  return bd_before(a, ia, b, ib);
}

__global__ void __launch_bounds__(1024) k_bd_chunk_sort(int64_t nn, int ch, const double* D, double* sk, int32_t* si) {
  __shared__ double key[kBdChunk];
  __shared__ int32_t idx[kBdChunk];
  const int64_t c0 = (int64_t)blockIdx.x * ch;
  for (int t = threadIdx.x; t < ch; t += blockDim.x) {
    const int64_t i = c0 + t;
    key[t] = i < nn ? D[i] : 0.0;
    idx[t] = (int32_t)(i < nn ? i : nn + t);
  }
  __syncthreads();
  for (int k = 2; k <= ch; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < ch / 2; t += blockDim.x) {
        const int lo = 2 * j * (t / j) + (t % j), hi = lo + j;
        const bool up = (lo & k) == 0;
        const bool swap = up ? bd_before_pad(key[hi], idx[hi], key[lo], idx[lo], nn)
                             : bd_before_pad(key[lo], idx[lo], key[hi], idx[hi], nn);
        if (swap) {
          const double kv = key[lo];
          key[lo] = key[hi];
          key[hi] = kv;
          const int32_t iv = idx[lo];
          idx[lo] = idx[hi];
          idx[hi] = iv;
        }
      }
      __syncthreads();
    }
  }
  for (int t = threadIdx.x; t < ch && c0 + t < nn; t += blockDim.x) {
    sk[c0 + t] = key[t];
    si[c0 + t] = idx[t];
  }
}

__global__ void __launch_bounds__(256) k_bd_rank(int64_t nn, int ch, const double* D, const double* z,
                                                const double* sk, const int32_t* si, double* Ds, double* zs,
                                                int32_t* perm) {
  const int64_t nch = (nn + ch - 1) / ch;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nn; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = q / ch;  // q: sorted place within chunk c
    const int32_t i = si[q];
    const double v = sk[q];
    int64_t rk = q - c * ch;
    for (int64_t c2 = 0; c2 < nch; ++c2) {
      if (c2 == c) continue;
      const int64_t b0 = c2 * ch, len = nn - b0 < ch ? nn - b0 : ch;
      int64_t lo = 0, hi = len;  // entries of chunk c2 before (v, i)
      while (lo < hi) {
        const int64_t m = (lo + hi) >> 1;
        if (bd_before(sk[b0 + m], si[b0 + m], v, i)) lo = m + 1;
        else hi = m;
      }
      rk += lo;
    }
    if (i < 0 || i >= nn || rk < 0 || rk >= nn) continue;  // cannot happen: a permutation
    Ds[rk] = D[i];
    if (z) zs[rk] = z[i];
    perm[rk] = i;
  }
}

// Deflation of one rank-one step over the sorted poles, by one block.  zs is normalised in
// place (rho = ||z||^2), tol = 8 eps max(|D|max, |z|max); type 1 deflates pole j when
// rho |z_j| <= tol.  Type 2 scans the survivors in order: the candidate p (the previous
// survivor, with its values as left by the scan) and the next survivor j give
// tau = hypot(z_j, z_p), c = z_j / tau, s = -z_p / tau; when |(D_j - D_p) c s| <= tol the
// rotation is recorded, z_j = tau, z_p = 0, both poles rotated, p deflated, else p is kept.
// The pairs are tested in parallel on the original values (valid whenever the previous
// pair did not rotate); one thread then resolves the chain, redoing a test only right after
// a rotation.  The outputs are those of the sequential scan: kept in scan order, rotations
// in order, defl in the order the scan deflates (keyed by the position being scanned),
// cnt = {K, nd, nrot}, *rho_out.  A non-finite pole or weight records TDC_ENONFINITE and
// deflates every pole (no secular solve and no product run on it).
constexpr int kBdDefThreads = 1024;
constexpr int64_t kBdDefMaxN = (int64_t)48 * 1024 * 8;  // two bit arrays in 96 KB of shared memory

__device__ __forceinline__ double block_sum_bd(double v, double* red) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];  // fixed order: reproducible
  return t;
}
__device__ __forceinline__ double block_max_bd(double v, double* red) {
  v = warp_max(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, red[w]);
  return t;
}
// exclusive prefix of f over the block (blockDim.x = kBdDefThreads) and the block's total
__device__ __forceinline__ int block_scan_bd(int f, int* wcnt, int& total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned m = __ballot_sync(0xffffffffu, f);
  __syncthreads();
  if (lane == 0) wcnt[wid] = __popc(m);
  __syncthreads();
  int before = 0;
  total = 0;
  for (int w = 0; w < kBdDefThreads / 32; ++w) {
    if (w < wid) before += wcnt[w];
    total += wcnt[w];
  }
  return before + __popc(m & ((1u << lane) - 1u));
}

__global__ void __launch_bounds__(kBdDefThreads) k_bd_deflate(int64_t nn, double* Ds, double* zs, int32_t* kept,
                                                             int32_t* defl, int32_t* rotp, double* rotcs,
                                                             int32_t* cnt, double* rho_out, BdScratch S,
                                                             int* status) {
  extern __shared__ unsigned rotbit[];  // speculative outcome of survivor pair (q - 1, q), then dbit
  __shared__ double red[32];
  __shared__ int wcnt[32];
  const int tid = threadIdx.x;
  double s2 = 0.0, dmax = 0.0;
  bool fin = true;
  for (int64_t i = tid; i < nn; i += blockDim.x) {
    s2 = fma(zs[i], zs[i], s2);
    dmax = fmax(dmax, fabs(Ds[i]));
    fin = fin && isfinite(zs[i]) && isfinite(Ds[i]);
  }
  const int bad = __syncthreads_or(!fin);
  s2 = block_sum_bd(s2, red);
  dmax = block_max_bd(dmax, red);
  if (bad || !isfinite(s2)) {
    if (tid == 0) set_status(status, TDC_ENONFINITE);
    for (int64_t i = tid; i < nn; i += blockDim.x) defl[i] = (int32_t)i;
    if (tid == 0) {
      cnt[0] = 0;
      cnt[1] = (int32_t)nn;
      cnt[2] = 0;
      *rho_out = 0.0;
    }
    return;
  }
  const double zn = sqrt(s2), rho = s2;
  double zmax = 0.0;
  for (int64_t i = tid; i < nn; i += blockDim.x) {
    double v = zs[i];
    if (zn > 0.0) v /= zn;
    zs[i] = v;
    zmax = fmax(zmax, fabs(v));
  }
  zmax = block_max_bd(zmax, red);
  const double tol = 8.0 * kBdEps * fmax(dmax, zmax);
  // type 1, and the survivors compacted in order
  int64_t M = 0;
  for (int64_t i0 = 0; i0 < nn; i0 += blockDim.x) {
    const int64_t i = i0 + tid;
    const bool t1 = i < nn && (!(zn > 0.0) || rho * fabs(zs[i]) <= tol);
    const bool sv = i < nn && !t1;
    int total = 0;
    const int pos = block_scan_bd(sv ? 1 : 0, wcnt, total);
    if (sv) S.surv[M + pos] = (int32_t)i;
    if (i < nn) S.slot[i] = t1 ? (int32_t)i : -1;
    M += total;
  }
  // type 2 on the original values, every consecutive survivor pair at once
  const int64_t nwords = (M + 31) / 32;
  unsigned* dbit = rotbit + (nn + 31) / 32;  // survivor q deflated by a rotation
  for (int64_t w = tid; w < nwords; w += blockDim.x) dbit[w] = 0u;
  for (int64_t q0 = 0; q0 < M; q0 += blockDim.x) {
    const int64_t q = q0 + tid;
    bool rot = false;
    if (q >= 1 && q < M) {
      const int32_t pa = S.surv[q - 1], pb = S.surv[q];
      const double zp = zs[pa], zj = zs[pb], dp = Ds[pa], dj = Ds[pb];
      const double w = hypot(zj, zp), t = dj - dp;
      const double c = zj / w, s = -zp / w;
      rot = fabs(t * c * s) <= tol;
      if (rot) {
        S.c[q] = c;
        S.s[q] = s;
        S.w[q] = w;
        S.dp[q] = dp * c * c + dj * s * s;
        S.dn[q] = dp * s * s + dj * c * c;
      }
    }
    const unsigned bits = __ballot_sync(0xffffffffu, rot);
    if ((tid & 31) == 0 && q < M) rotbit[q >> 5] = bits;
  }
  __syncthreads();
  // the chain, in one thread: a pair whose candidate was left unchanged takes its
  // speculative outcome, so the scan jumps from one speculative rotation to the next and
  // evaluates a pair itself only right after a rotation
  if (tid == 0) {
    int32_t nr = 0;
    bool mod = false;  // the candidate's values were changed by the previous rotation
    double zc = 0.0, dc = 0.0;
    int64_t q = 1;
    while (q < M) {
      bool rot;
      double c = 0.0, s = 0.0, w = 0.0, dp = 0.0, dn = 0.0;
      if (!mod) {
        int64_t wd = q >> 5;
        unsigned bits = rotbit[wd] & (0xffffffffu << (q & 31));
        while (bits == 0u && ++wd < nwords) bits = rotbit[wd];
        if (bits == 0u) break;
        q = wd * 32 + (__ffs(bits) - 1);
        if (q >= M) break;
        rot = true;
        c = S.c[q];
        s = S.s[q];
        w = S.w[q];
        dp = S.dp[q];
        dn = S.dn[q];
      } else {
        const int32_t pb = S.surv[q];
        const double zj = zs[pb], dj = Ds[pb];
        w = hypot(zj, zc);
        const double t = dj - dc;
        c = zj / w;
        s = -zc / w;
        rot = fabs(t * c * s) <= tol;
        if (rot) {
          dp = dc * c * c + dj * s * s;
          dn = dc * s * s + dj * c * c;
        }
      }
      if (rot) {
        const int32_t pa = S.surv[q - 1], pb = S.surv[q];
        zs[pb] = w;
        zs[pa] = 0.0;
        Ds[pa] = dp;
        Ds[pb] = dn;
        rotp[2 * nr] = pa;
        rotp[2 * nr + 1] = pb;
        rotcs[2 * nr] = c;
        rotcs[2 * nr + 1] = s;
        ++nr;
        S.slot[pb] = pa;
        dbit[(q - 1) >> 5] |= 1u << ((q - 1) & 31);
        mod = true;
        zc = w;
        dc = dn;
      } else {
        mod = false;
      }
      ++q;
    }
    cnt[2] = nr;
    *rho_out = rho;
  }
  __syncthreads();
  // kept: the survivors no rotation deflated, in order
  int64_t K = 0;
  for (int64_t q0 = 0; q0 < M; q0 += blockDim.x) {
    const int64_t q = q0 + tid;
    const bool kp = q < M && !((dbit[q >> 5] >> (q & 31)) & 1u);
    int total = 0;
    const int pos = block_scan_bd(kp ? 1 : 0, wcnt, total);
    if (kp) kept[K + pos] = S.surv[q];
    K += total;
  }
  if (tid == 0) cnt[0] = (int32_t)K;
  // deflated entries in scan order
  int64_t nd = 0;
  for (int64_t i0 = 0; i0 < nn; i0 += blockDim.x) {
    const int64_t i = i0 + tid;
    const int32_t e = i < nn ? S.slot[i] : -1;
    int total = 0;
    const int pos = block_scan_bd(e >= 0 ? 1 : 0, wcnt, total);
    if (e >= 0) defl[nd + pos] = e;
    nd += total;
  }
  if (tid == 0) cnt[1] = (int32_t)nd;
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
cudaError_t launch_bd_leaf_trd(const BdLeafArgs& A, const BdLeafTable& T, cudaStream_t s) {
  if (A.nleaf <= 0) return cudaSuccess;
  k_bd_leaf_trd<<<(unsigned)A.nleaf, kBdLeafThreads, 0, s>>>(A, T);
  return cudaGetLastError();
}
cudaError_t launch_bd_leaf_back(const BdLeafArgs& A, const BdLeafTable& T, cudaStream_t s) {
  if (A.nleaf <= 0) return cudaSuccess;
  k_bd_leaf_back<<<(unsigned)A.nleaf, kBdLeafThreads, 0, s>>>(A, T);
  return cudaGetLastError();
}
cudaError_t launch_bd_z(int64_t nn, const double* Q, int64_t ldq, int64_t ra, int64_t rb, int b, const double* w,
                        double* z, cudaStream_t s) {
  k_bd_z<<<grid_for(nn), 256, 0, s>>>(nn, Q, ldq, ra, rb, b, w, z);
  return cudaGetLastError();
}
cudaError_t launch_bd_sort(int64_t nn, const double* D, const double* z, double* Ds, double* zs, int32_t* perm,
                           const BdScratch& S, cudaStream_t s) {
  if (nn <= 0) return cudaSuccess;
  int ch = 2;
  while (ch < kBdChunk && ch < nn) ch <<= 1;
  k_bd_chunk_sort<<<(unsigned)((nn + ch - 1) / ch), std::max(32, std::min(1024, ch / 2)), 0, s>>>(nn, ch, D, S.sk,
                                                                                                 S.si);
  k_bd_rank<<<grid_for(nn), 256, 0, s>>>(nn, ch, D, z, S.sk, S.si, Ds, zs, perm);
  return cudaGetLastError();
}
cudaError_t launch_bd_deflate(int64_t nn, double* Ds, double* zs, int32_t* kept, int32_t* defl, int32_t* rotp,
                              double* rotcs, int32_t* cnt, double* rho, const BdScratch& S, int* status,
                              cudaStream_t s) {
  if (nn > kBdDefMaxN) return cudaErrorInvalidValue;
  const size_t smem = 2 * sizeof(unsigned) * (size_t)((std::max<int64_t>(nn, 1) + 31) / 32);
  static bool attr[64] = {false};  // once per device
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!attr[dev]) {
    e = cudaFuncSetAttribute(k_bd_deflate, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    if (e != cudaSuccess) return e;
    attr[dev] = true;
  }
  k_bd_deflate<<<1, kBdDefThreads, smem, s>>>(nn, Ds, zs, kept, defl, rotp, rotcs, cnt, rho, S, status);
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
