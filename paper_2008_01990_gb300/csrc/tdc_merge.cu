// tdc_merge.cu -- the merge step of Cuppen's divide and conquer on the GPU,
// level by level over every node of every problem in the plan:
//   k_dmod      corner modification of the split points (Eq. (T2))
//   k_leaf      leaf eigensolves (Algorithm 1, "QR"): two warps per leaf, or
//   k_leaf_multi  a lane per leaf for leaves of at most 32 rows
//   k_prepare   z (Eq. (T3)) from the children's boundary rows, merge of the
//               two sorted spectra, deflation scan (Section 3.2, Eq. (T3-def)),
//               compaction
//   k_boundary_rot  the children's boundary rows through the deflating rotations
//   k_rotate    plane rotations of deflation applied to Q's columns
//   k_secular   secular equation (Eq. (secular)), one warp per root (a thread
//               per root for small merges on many-merge levels), FP64, roots
//               stored as (origin pole, offset) (Eq. (d-lambda))
//   k_lowner    zhat recomputed from (d, lambda), one warp (or thread) per pole
//   k_colnorm   normalisers s_j of the Cauchy-like Qhat (Eq. (Q_Cauchy)) and,
//               below the top level, the node's boundary rows
//   k_finalize  ascending order of all eigenvalues of the node, column targets
//   k_boundary_out  boundary rows in output order
//   k_copy_defl deflated eigenvectors copied to their columns
//   k_sign_out  sign convention and eigenvalue output
#include <float.h>
#include <math.h>

#include "tdc_common.cuh"

namespace tdc {

static constexpr double kEps = DBL_EPSILON;

// ---------------------------------------------------------------------------
// corner modification: every split point p (a leaf boundary) subtracts |e|
// from the diagonal entries on both sides
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool is_boundary(int64_t r, int64_t n, int t) {
  if (r <= 0 || r >= n) return false;
  int64_t i = ((r << t) + n - 1) / n;  // ceil(r 2^t / n)
  return ((i * n) >> t) == r;
}

__global__ void k_dmod(Plan P) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < P.nslots;
       s += (int64_t)gridDim.x * blockDim.x) {
    int pi = find_problem_by_slot(P.prob, P.nprob, s);
    const Problem& p = P.prob[pi];
    int64_t r = s - p.voff;
    const double d0 = P.d[p.off_de + r];
    bool ok = isfinite(d0);
    if (r + 1 < p.n) ok = ok && isfinite(P.e[p.off_de + r]);
    double d = input_entry(d0, p.escale);
    if (is_boundary(r, p.n, p.depth)) d -= fabs(input_entry(P.e[p.off_de + r - 1], p.escale));
    if (is_boundary(r + 1, p.n, p.depth)) d -= fabs(input_entry(P.e[p.off_de + r], p.escale));
    if (!ok) set_status(P.status, TDC_ENONFINITE);
    P.v.dmod[s] = d;
  }
}

// Each problem's input scale (a block per problem): the largest finite |d|, |e|, and
// escale = its binary exponent when that lies outside [2^-400, 2^400], else 0.
__global__ void __launch_bounds__(256) k_input_scale(Plan P) {
  __shared__ double red[8];
  for (int pi = blockIdx.x; pi < P.nprob; pi += gridDim.x) {
    const Problem& p = P.prob[pi];
    double m = 0.0;
    for (int64_t r = threadIdx.x; r < p.n; r += blockDim.x) {
      m = fmax(m, fabs(finite_or_zero(P.d[p.off_de + r])));
      if (r + 1 < p.n) m = fmax(m, fabs(finite_or_zero(P.e[p.off_de + r])));
    }
    m = warp_max(m);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
      m = fmax(m, red[0]);
      const bool out = m > 0x1p400 || (m > 0.0 && m < 0x1p-400);
      const_cast<Problem*>(P.prob)[pi].escale = out ? ilogb(m) : 0;
    }
  }
}

cudaError_t launch_dmod(const Plan& P, cudaStream_t s) {
  if (P.nslots == 0) return cudaSuccess;
  k_input_scale<<<(unsigned)std::min<int64_t>(P.nprob, 152 * 8), 256, 0, s>>>(P);
  int64_t blocks = (P.nslots + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_dmod<<<(unsigned)blocks, 256, 0, s>>>(P);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Leaf eigensolves: implicit symmetric QR with Wilkinson shift on an L x L
// tridiagonal (L <= 64), one warp per leaf.  Lane 0 runs the scalar sweep and
// records its rotations; all lanes then apply them to their rows of Q, which
// lives column-major in shared memory.
// ---------------------------------------------------------------------------
static constexpr int kMaxLeaf = 64;

// One leaf per block of two warps.  Implicit symmetric QR with Wilkinson shift:
// warp 0 tests every off-diagonal for negligibility in parallel (one ballot finds
// the active block [pp, q]) and lane 0 chases the bulge through it, carrying the
// running diagonal / off-diagonal entries in registers; warp 1 meanwhile applies
// the previous sweep's rotations to the eigenvector block (two rows per lane,
// the running column in a register).  The rotations of consecutive sweeps are
// double-buffered, so the sequential chase and the parallel update overlap.
__global__ void __launch_bounds__(64) k_leaf(Plan P, int64_t nleaves) {
  extern __shared__ double sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int64_t g = blockIdx.x;
  if (g >= nleaves) return;
  // problem owning global leaf g (problems sorted by leaf0 ascending)
  int lo_i = 0, hi_i = P.nprob - 1;
  while (lo_i < hi_i) {
    int m = (lo_i + hi_i + 1) >> 1;
    if (P.prob[m].leaf0 <= g) lo_i = m; else hi_i = m - 1;
  }
  const Problem& p = P.prob[lo_i];
  int64_t li = g - p.leaf0;
  int t = p.depth;
  int64_t lo = node_bound(li, p.n, t), hi = node_bound(li + 1, p.n, t);
  const int L = (int)(hi - lo);
  double* Qs = sm;                 // L*L, column-major
  double* dd = Qs + L * L;         // L
  double* ee = dd + L;             // L
  double* cs = ee + L;             // 2 buffers x 2L (c, s of each rotation)
  int* ctrl = (int*)(cs + 4 * L);  // [b][0..1] = pp, q of the sweep in buffer b; [4] = done
  int* perm = ctrl + 6;            // L
  for (int k = tid; k < L * L; k += blockDim.x) Qs[k] = ((k % L) == (k / L)) ? 1.0 : 0.0;
  for (int k = tid; k < L; k += blockDim.x) {
    dd[k] = P.v.dmod[p.voff + lo + k];
    ee[k] = (k < L - 1) ? input_entry(P.e[p.off_de + lo + k], p.escale) : 0.0;
  }
  if (tid == 0) ctrl[4] = (L <= 1) ? 1 : 0;
  __syncthreads();
  const int max_sweeps = 40 * (L > 0 ? L : 1);
  int sweep = 0;
  while (!ctrl[4]) {
    const int b = sweep & 1;
    if (warp == 0) {
      // negligible off-diagonals (all lanes), then the trailing unreduced block
      unsigned long long nz = 0ull;
      for (int h = 0; h < 2; ++h) {
        const int k = lane + 32 * h;
        bool keep = false;
        if (k < L - 1) {
          const double ek = ee[k];
          if (fabs(ek) <= kEps * (fabs(dd[k]) + fabs(dd[k + 1]))) ee[k] = 0.0;
          else keep = ek != 0.0;
        }
        nz |= (unsigned long long)__ballot_sync(0xffffffffu, keep) << (32 * h);
      }
      __syncwarp();
      if (lane == 0) {
        if (nz == 0ull) {
          ctrl[4] = 1;
          ctrl[2 * b] = 0;
          ctrl[2 * b + 1] = 0;
        } else if (sweep >= max_sweeps) {
          ctrl[4] = 1;
          ctrl[2 * b] = 0;
          ctrl[2 * b + 1] = 0;
          set_status(P.status, TDC_ENOCONV);
        } else {
          const int q = 64 - __clzll((long long)nz);  // ee[q-1] != 0, ee[q..] == 0
          const unsigned long long below = (q - 1 > 0) ? (~nz & ((1ull << (q - 1)) - 1ull)) : 0ull;
          const int pp = below ? 64 - __clzll((long long)below) : 0;
          // Wilkinson shift: eigenvalue of the trailing 2x2 block nearer to dd[q]
          const double hd = 0.5 * (dd[q - 1] - dd[q]);
          const double bq = ee[q - 1];
          const double hh = hypot(hd, bq);
          const double mu = dd[q] - bq * bq / (hd + copysign(hh, hd));
          double a0 = dd[pp], bk = ee[pp];
          double x = a0 - mu, y = bk;
          double* cb = cs + 2 * L * b;
          for (int k = pp; k < q; ++k) {
            const double a1 = dd[k + 1];
            const double en = (k < q - 1) ? ee[k + 1] : 0.0;
            // Givens rotation from (x, y) through a refined reciprocal square root
            // (no division on the sequential path); hypot only where squares leave range
            const double t2 = fma(x, x, y * y);
            double r, c = 1.0, sn = 0.0;
            if (t2 > 1e-290 && t2 < 1e290) {
              const double ri = rsqrt_nr(t2);
              c = x * ri; sn = y * ri; r = t2 * ri;
            } else {
              r = hypot(x, y);
              if (r != 0.0) { c = x / r; sn = y / r; }
            }
            if (k > pp) ee[k - 1] = r;
            const double cc = c * c, ss = sn * sn, c2s = 2.0 * c * sn * bk;
            dd[k] = cc * a0 + c2s + ss * a1;
            const double a0n = ss * a0 - c2s + cc * a1;
            const double ek = c * sn * (a1 - a0) + (cc - ss) * bk;
            if (k < q - 1) {
              y = sn * en;
              bk = c * en;
              x = ek;
            } else {
              ee[k] = ek;
            }
            a0 = a0n;
            cb[2 * k] = c;
            cb[2 * k + 1] = sn;
          }
          dd[q] = a0;
          ctrl[2 * b] = pp;
          ctrl[2 * b + 1] = q;
        }
      }
    } else if (sweep > 0) {
      // rotations of the previous sweep, rows lane and lane + 32
      const int pb = b ^ 1;
      const int pp = ctrl[2 * pb], q = ctrl[2 * pb + 1];
      const double* cb = cs + 2 * L * pb;
      const int r0 = lane, r1 = lane + 32;
      if (r0 < L && q > pp) {
        const bool two = r1 < L;
        double v0 = Qs[r0 + pp * L], v1 = two ? Qs[r1 + pp * L] : 0.0;
        for (int k = pp; k < q; ++k) {
          const double c = cb[2 * k], sn = cb[2 * k + 1];
          const double w0 = Qs[r0 + (k + 1) * L];
          Qs[r0 + k * L] = c * v0 + sn * w0;
          v0 = c * w0 - sn * v0;
          if (two) {
            const double w1 = Qs[r1 + (k + 1) * L];
            Qs[r1 + k * L] = c * v1 + sn * w1;
            v1 = c * w1 - sn * v1;
          }
        }
        Qs[r0 + q * L] = v0;
        if (two) Qs[r1 + q * L] = v1;
      }
    }
    __syncthreads();
    ++sweep;
  }
  // the sweep in the last buffer (if any) is still to be applied
  if (warp == 1 && sweep > 0) {
    const int pb = (sweep - 1) & 1;
    const int pp = ctrl[2 * pb], q = ctrl[2 * pb + 1];
    const double* cb = cs + 2 * L * pb;
    for (int r = lane; r < L && q > pp; r += 32) {
      double v = Qs[r + pp * L];
      for (int k = pp; k < q; ++k) {
        const double c = cb[2 * k], sn = cb[2 * k + 1];
        const double w = Qs[r + (k + 1) * L];
        Qs[r + k * L] = c * v + sn * w;
        v = c * w - sn * v;
      }
      Qs[r + q * L] = v;
    }
  }
  __syncthreads();
  // ascending order (stable): rank of each eigenvalue
  for (int k = tid; k < L; k += blockDim.x) {
    const double v = dd[k];
    int rk = 0;
    for (int m = 0; m < L; ++m) {
      const double w = dd[m];
      rk += (w < v || (w == v && m < k)) ? 1 : 0;
    }
    perm[rk] = k;
  }
  __syncthreads();
  double* dst;
  int64_t ld;
  if (t & 1) { dst = P.Q1 + p.qoff1; ld = p.n; }
  else { dst = P.Q0 + p.off_q; ld = p.ld0; }
  dst += lo + lo * ld;
  for (int k = 0; k < L; ++k) {
    int c = perm[k];
    for (int r = tid; r < L; r += blockDim.x) dst[r + k * ld] = Qs[r + c * L];
  }
  const int par = t & 1;
  for (int k = tid; k < L; k += blockDim.x) {
    P.lam2[par][p.voff + lo + k] = dd[perm[k]];
    P.bf2[par][p.voff + lo + k] = Qs[perm[k] * L];
    P.bl2[par][p.voff + lo + k] = Qs[(L - 1) + perm[k] * L];
  }
}

// Many small leaves per block.  The sequential bulge chase costs one warp
// instruction per FP64 operation whether one lane or 32 are active, so here lane l
// of warp 0 runs the whole QR iteration of leaf l (its own deflation scan, shift
// and chase) and the G leaves of the block advance together; warps 1.. apply each
// round's rotations to the leaves' eigenvector blocks (one row per lane, the
// rotations of consecutive rounds double-buffered).  Used when leaves have at
// most 32 rows; every leaf gets the same arithmetic as in k_leaf.
__global__ void __launch_bounds__(1024) k_leaf_multi(Plan P, int64_t nleaves, int Lm, int G) {
  extern __shared__ double sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int slot = Lm * Lm + 6 * Lm;  // doubles per leaf: Q block, d, e, 2 x (c, s) buffers
  int* ib = reinterpret_cast<int*>(sm + (size_t)G * slot);
  int* ctrl = ib;                  // [G][4]: pp, q of buffers 0 and 1
  int* perm = ctrl + 4 * G;        // [G][Lm]
  int* sL = perm + G * Lm;         // [G] leaf order (0: no leaf)
  int* sprob = sL + G;             // [G] problem index
  long long* slo = reinterpret_cast<long long*>(sprob + G + ((6 * G + G * Lm) & 1));  // [G] first row
  const int64_t g0 = (int64_t)blockIdx.x * G;
  if (tid < G) {
    const int64_t g = g0 + tid;
    int L = 0, pi = 0;
    long long lo = 0;
    if (g < nleaves) {
      int a = 0, b = P.nprob - 1;
      while (a < b) {
        const int m = (a + b + 1) >> 1;
        if (P.prob[m].leaf0 <= g) a = m; else b = m - 1;
      }
      const Problem& pr = P.prob[a];
      const int64_t li = g - pr.leaf0;
      lo = node_bound(li, pr.n, pr.depth);
      L = (int)(node_bound(li + 1, pr.n, pr.depth) - lo);
      pi = a;
    }
    sL[tid] = L;
    sprob[tid] = pi;
    slo[tid] = lo;
  }
  __syncthreads();
  for (int x = tid; x < G * Lm * Lm; x += blockDim.x) {
    const int l = x / (Lm * Lm), k = x % (Lm * Lm);
    sm[(size_t)l * slot + k] = ((k % Lm) == (k / Lm)) ? 1.0 : 0.0;
  }
  for (int x = tid; x < G * Lm; x += blockDim.x) {
    const int l = x / Lm, k = x % Lm, L = sL[l];
    double* dd = sm + (size_t)l * slot + Lm * Lm;
    double* ee = dd + Lm;
    if (k < L) {
      const Problem& pr = P.prob[sprob[l]];
      dd[k] = P.v.dmod[pr.voff + slo[l] + k];
      ee[k] = (k < L - 1) ? input_entry(P.e[pr.off_de + slo[l] + k], pr.escale) : 0.0;
    }
  }
  __syncthreads();
  const int lpw = 32 / Lm;                 // leaves per apply warp
  const int max_sweeps = 40 * (Lm > 0 ? Lm : 1);
  int sweeps = 0;
  bool done = !(warp == 0 && lane < G && sL[lane] > 1);
  for (int round = 0;; ++round) {
    const int b = round & 1;
    bool nonempty = false;
    if (warp == 0) {
      if (lane < G) {
        const int L = sL[lane];
        double* dd = sm + (size_t)lane * slot + Lm * Lm;
        double* ee = dd + Lm;
        double* cb = ee + Lm + 2 * Lm * b;
        int pp = 0, q = 0;
        if (!done) {
          q = L - 1;
          for (int k = 0; k < q; ++k)
            if (fabs(ee[k]) <= kEps * (fabs(dd[k]) + fabs(dd[k + 1]))) ee[k] = 0.0;
          while (q > 0 && ee[q - 1] == 0.0) --q;
          if (q == 0) {
            done = true;
          } else if (sweeps >= max_sweeps) {
            done = true;
            q = 0;
            set_status(P.status, TDC_ENOCONV);
          } else {
            ++sweeps;
            pp = q - 1;
            while (pp > 0 && ee[pp - 1] != 0.0) --pp;
            const double hd = 0.5 * (dd[q - 1] - dd[q]);
            const double bq = ee[q - 1];
            const double hh = hypot(hd, bq);
            const double mu = dd[q] - bq * bq / (hd + copysign(hh, hd));
            double a0 = dd[pp], bk = ee[pp];
            double x = a0 - mu, y = bk;
            for (int k = pp; k < q; ++k) {
              const double a1 = dd[k + 1];
              const double en = (k < q - 1) ? ee[k + 1] : 0.0;
              const double t2 = fma(x, x, y * y);
              double r, c = 1.0, sn = 0.0;
              if (t2 > 1e-290 && t2 < 1e290) {
                const double ri = rsqrt_nr(t2);
                c = x * ri; sn = y * ri; r = t2 * ri;
              } else {
                r = hypot(x, y);
                if (r != 0.0) { c = x / r; sn = y / r; }
              }
              if (k > pp) ee[k - 1] = r;
              const double cc = c * c, ss = sn * sn, c2s = 2.0 * c * sn * bk;
              dd[k] = cc * a0 + c2s + ss * a1;
              const double a0n = ss * a0 - c2s + cc * a1;
              const double ek = c * sn * (a1 - a0) + (cc - ss) * bk;
              if (k < q - 1) {
                y = sn * en;
                bk = c * en;
                x = ek;
              } else {
                ee[k] = ek;
              }
              a0 = a0n;
              cb[2 * k] = c;
              cb[2 * k + 1] = sn;
            }
            dd[q] = a0;
            nonempty = true;
          }
        }
        ctrl[4 * lane + 2 * b] = nonempty ? pp : 0;
        ctrl[4 * lane + 2 * b + 1] = nonempty ? q : 0;
      }
    } else if (round > 0) {
      // rotations of the previous round: apply warp w takes leaves (w-1)*lpw .. + lpw - 1
      const int l = (warp - 1) * lpw + lane / Lm, r = lane % Lm;
      if (lane < lpw * Lm && l < G && r < sL[l]) {
        const int pb = b ^ 1;
        const int pp = ctrl[4 * l + 2 * pb], q = ctrl[4 * l + 2 * pb + 1];
        if (q > pp) {
          double* Qs = sm + (size_t)l * slot;
          const double* cb = Qs + Lm * Lm + 2 * Lm + 2 * Lm * pb;
          double v = Qs[r + pp * Lm];
          for (int k = pp; k < q; ++k) {
            const double c = cb[2 * k], sn = cb[2 * k + 1];
            const double w = Qs[r + (k + 1) * Lm];
            Qs[r + k * Lm] = c * v + sn * w;
            v = c * w - sn * v;
          }
          Qs[r + q * Lm] = v;
        }
      }
    }
    if (!__syncthreads_or(nonempty ? 1 : 0)) break;
  }
  // ascending order (stable) per leaf, then the blocks and eigenvalues out
  for (int x = tid; x < G * Lm; x += blockDim.x) {
    const int l = x / Lm, k = x % Lm, L = sL[l];
    if (k >= L) continue;
    const double* dd = sm + (size_t)l * slot + Lm * Lm;
    const double v = dd[k];
    int rk = 0;
    for (int m = 0; m < L; ++m) {
      const double w = dd[m];
      rk += (w < v || (w == v && m < k)) ? 1 : 0;
    }
    perm[l * Lm + rk] = k;
  }
  __syncthreads();
  for (int x = tid; x < G * Lm * Lm; x += blockDim.x) {
    const int l = x / (Lm * Lm), rem = x % (Lm * Lm), k = rem / Lm, r = rem % Lm, L = sL[l];
    if (k >= L || r >= L) continue;
    const Problem& pr = P.prob[sprob[l]];
    double* dst;
    int64_t ld;
    if (pr.depth & 1) { dst = P.Q1 + pr.qoff1; ld = pr.n; }
    else { dst = P.Q0 + pr.off_q; ld = pr.ld0; }
    const int64_t lo = slo[l];
    dst[(lo + r) + (lo + k) * ld] = sm[(size_t)l * slot + r + perm[l * Lm + k] * Lm];
  }
  for (int x = tid; x < G * Lm; x += blockDim.x) {
    const int l = x / Lm, k = x % Lm, L = sL[l];
    if (k >= L) continue;
    const Problem& pr = P.prob[sprob[l]];
    const int par = pr.depth & 1, c = perm[l * Lm + k];
    const int64_t o = pr.voff + slo[l] + k;
    P.lam2[par][o] = sm[(size_t)l * slot + Lm * Lm + c];
    P.bf2[par][o] = sm[(size_t)l * slot + c * Lm];
    P.bl2[par][o] = sm[(size_t)l * slot + (L - 1) + c * Lm];
  }
}

cudaError_t launch_leaves(const Plan& P, int64_t nleaves, int max_leaf, cudaStream_t s) {
  if (nleaves == 0) return cudaSuccess;
  if (max_leaf > kMaxLeaf) return cudaErrorInvalidValue;
  if (max_leaf <= 32 && nleaves >= 64) {
    // G leaves per block within a shared-memory budget, one apply warp per 32 rows
    const int Lm = max_leaf;
    // per leaf: Q block, d, e and two rotation buffers; pp/q of both buffers, the
    // permutation, order, problem and first row
    const size_t per = sizeof(double) * (size_t)(Lm * Lm + 6 * Lm) + sizeof(int) * (size_t)(6 + Lm) + 8;
    const int lpw = 32 / Lm;
    int G = (int)std::min<size_t>(32, (size_t)(96 * 1024) / per);
    G = std::max(1, std::min(G, 31 * lpw));
    const int warps = 1 + (G + lpw - 1) / lpw;
    const size_t smem = per * G + 64;
    cudaError_t e = cudaFuncSetAttribute(k_leaf_multi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_leaf_multi<<<(unsigned)((nleaves + G - 1) / G), 32 * warps, smem, s>>>(P, nleaves, Lm, G);
    return cudaGetLastError();
  }
  size_t smem = sizeof(double) * (max_leaf * max_leaf + 6 * max_leaf) + sizeof(int) * (6 + max_leaf);
  k_leaf<<<(unsigned)nleaves, 64, smem, s>>>(P, nleaves);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Block helpers
// ---------------------------------------------------------------------------
template <typename T>
__device__ T block_reduce_max(T v, T* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    T m = red[0];
    for (int i = 1; i < nw; ++i) m = max(m, red[i]);
    red[0] = m;
  }
  __syncthreads();
  T r = red[0];
  __syncthreads();
  return r;
}

// exclusive prefix of per-thread counts (a, b) across the block
__device__ void block_excl_scan2(int& a, int& b, int* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  int ia = a, ib = b;
  for (int o = 1; o < 32; o <<= 1) {
    int ta = __shfl_up_sync(0xffffffffu, ia, o), tb = __shfl_up_sync(0xffffffffu, ib, o);
    if (lane >= o) { ia += ta; ib += tb; }
  }
  __syncthreads();
  if (lane == 31) { red[2 * w] = ia; red[2 * w + 1] = ib; }
  __syncthreads();
  if (threadIdx.x == 0) {
    int sa = 0, sb = 0;
    for (int i = 0; i < nw; ++i) {
      int ta = red[2 * i], tb = red[2 * i + 1];
      red[2 * i] = sa; red[2 * i + 1] = sb;
      sa += ta; sb += tb;
    }
  }
  __syncthreads();
  a = red[2 * w] + ia - a;
  b = red[2 * w + 1] + ib - b;
  __syncthreads();
}

// ---------------------------------------------------------------------------
// k_prepare: one block per merge.
// ---------------------------------------------------------------------------

// Type-2 deflation test of pole (D, z) against the last kept pole (pD, pz):
// |(D - pD) c s| <= tol with c s = -z pz / (z^2 + pz^2), i.e. without division or
// root.  Every rounding is explicit so that the speculative (parallel) and the
// sequential evaluation of the same pair give the same answer.
__device__ __forceinline__ bool type2_test(double D, double z, double pD, double pz, double tol) {
  const double t2 = __fma_rn(z, z, __dmul_rn(pz, pz));
  return fabs(__dmul_rn(__dmul_rn(__dsub_rn(D, pD), z), pz)) <= __dmul_rn(tol, t2);
}

// The rotation that moves all of z onto the new pole: c = z/tau, s = -pz/tau,
// tau = hypot(z, pz); the deflated value dp and the survivor's new value di.
__device__ __forceinline__ void type2_rot(double D, double z, double pD, double pz, double& cc, double& ss,
                                          double& tau, double& dp, double& di) {
  const double t2 = __fma_rn(z, z, __dmul_rn(pz, pz));
  const double r = rsqrt_nr(t2);
  cc = __dmul_rn(z, r);
  ss = __dmul_rn(-pz, r);
  tau = __dmul_rn(t2, r);
  const double c2 = __dmul_rn(cc, cc), s2 = __dmul_rn(ss, ss);
  dp = __fma_rn(pD, c2, __dmul_rn(D, s2));
  di = __fma_rn(pD, s2, __dmul_rn(D, c2));
}

__global__ void __launch_bounds__(1024) k_prepare(Plan P, int level) {
  __shared__ double redd[64];
  __shared__ int redi[64];
  __shared__ int sres[4];
  const int64_t g = blockIdx.x;
  const Node nd = make_node(P, level, g);
  const int n = (int)(nd.hi - nd.lo), n1 = (int)(nd.mid - nd.lo);
  const int64_t v0 = nd.v0;
  const Vecs& V = P.v;
  const double rho = 2.0 * fabs(nd.b);
  const double sg = nd.b < 0.0 ? -1.0 : 1.0;
  const double rs2 = 0.70710678118654752440;
  // 1. z: the last row of Q1 and the first row of Q2, the boundary rows the children
  //    left (the rows of their eigenvector matrices, kept apart so that this level
  //    does not have to wait for the children's full products)
  double mx = 0.0;
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    double D = P.clam[v0 + c];
    double z = (c < n1) ? P.cbl[v0 + c] : sg * P.cbf[v0 + c];
    z *= rs2;
    V.Dc[v0 + c] = D;
    V.zc[v0 + c] = z;
    mx = fmax(mx, fmax(fabs(D), fabs(z)));
  }
  const double tol = 8.0 * kEps * block_reduce_max(mx, redd);
  // 2. ascending order of the two sorted spectra (stable: first half first on ties)
  const double* D1 = P.clam + v0;
  const double* D2 = P.clam + v0 + n1;
  const int n2 = n - n1;
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  auto rank_of = [&](int c) -> int {
    const double D = P.clam[v0 + c];
    if (c < n1) {  // count of D2 < D
      int a = 0, b = n2;
      while (a < b) { int m = (a + b) >> 1; if (D2[m] < D) a = m + 1; else b = m; }
      return c + a;
    }
    int a = 0, b = n1;  // count of D1 <= D
    while (a < b) { int m = (a + b) >> 1; if (D1[m] <= D) a = m + 1; else b = m; }
    return (c - n1) + a;
  };
  for (int c = threadIdx.x; c < n; c += blockDim.x) V.perm[v0 + rank_of(c)] = c;
  __syncthreads();
  // the ranks form a permutation unless the spectra are not ordered (non-finite
  // values); then fall back to the identity so that every index stays in range
  for (int c = threadIdx.x; c < n; c += blockDim.x)
    if (V.perm[v0 + rank_of(c)] != c) s_bad = 1;
  __syncthreads();
  if (s_bad) {
    for (int c = threadIdx.x; c < n; c += blockDim.x) V.perm[v0 + c] = c;
    if (threadIdx.x == 0) set_status(P.status, TDC_ENONFINITE);
  }
  __syncthreads();
  // 3. deflation (Section 3.2).  Type 1 is a per-pole test; type 2 compares each
  //    remaining pole with the last kept one, which is sequential only through
  //    chains of rotations.  3a/3b run in parallel: the compacted list L of the
  //    poles that survive type 1, and for each consecutive pair of L the type-2 test
  //    and rotation evaluated on the original values (valid whenever the previous
  //    pair did not rotate).  3c resolves the sequence in one thread and does FP64
  //    work only right after a rotation.
  int* Lpos = P.v.stag + 2 * v0;    // sorted positions of the poles surviving type 1
  uint8_t* flag = P.v.cseg + v0;    // speculative type-2 outcome for pair (q-1, q)
  double* spc = P.v.skey + 2 * v0;  // speculative c (q) and s (n + q)
  double* sdp = P.v.Ds + v0;        // speculative deflated value of the predecessor
  double* sdi = P.v.zs + v0;        // speculative new value of the survivor
  double* stau = P.v.tau + v0;      // speculative new z of the survivor
  // 3a. type-1 entries go straight to the deflated list (sorted order), the rest to L
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int p0 = min(n, (int)threadIdx.x * per), p1 = min(n, p0 + per);
  int c_keep = 0, c_t1 = 0;
  for (int p = p0; p < p1; ++p) {
    const int c = V.perm[v0 + p];
    if (rho * fabs(V.zc[v0 + c]) <= tol) ++c_t1; else ++c_keep;
  }
  int o_keep = c_keep, o_t1 = c_t1;
  block_excl_scan2(o_keep, o_t1, redi);
  for (int p = p0; p < p1; ++p) {
    const int c = V.perm[v0 + p];
    if (rho * fabs(V.zc[v0 + c]) <= tol) {
      V.dcol[v0 + o_t1] = c;
      V.dval[v0 + o_t1] = V.Dc[v0 + c];
      V.dseg[v0 + o_t1] = (uint8_t)((c < n1) ? 1 : 2);
      ++o_t1;
    } else {
      Lpos[o_keep++] = p;
    }
  }
  if (threadIdx.x == blockDim.x - 1) { sres[0] = o_keep; sres[1] = o_t1; }
  __syncthreads();
  const int nL = sres[0], t1 = sres[1];
  __syncthreads();
  // 3b. speculative type-2 test and rotation for each consecutive pair of L
  //     (bit 0 of flag[q]), and for the pole after a speculative rotation the test
  //     against the rotated survivor (bit 1), which covers isolated pairs of
  //     equal poles without sequential FP64 work
  for (int q = 1 + threadIdx.x; q < nL; q += blockDim.x) {
    const int a = V.perm[v0 + Lpos[q - 1]], b = V.perm[v0 + Lpos[q]];
    const double pD = V.Dc[v0 + a], pz = V.zc[v0 + a];
    const double D = V.Dc[v0 + b], z = V.zc[v0 + b];
    const bool f = type2_test(D, z, pD, pz, tol);
    flag[q] = f ? 1 : 0;
    if (f) type2_rot(D, z, pD, pz, spc[q], spc[n + q], stau[q], sdp[q], sdi[q]);
  }
  __syncthreads();
  for (int q = 2 + threadIdx.x; q < nL; q += blockDim.x) {
    if (!(flag[q - 1] & 1)) continue;
    const int b = V.perm[v0 + Lpos[q]];
    if (type2_test(V.Dc[v0 + b], V.zc[v0 + b], sdi[q - 1], stau[q - 1], tol)) flag[q] |= 2;
  }
  __syncthreads();
  // 3c. resolution of the scan, pipelined over chunks of kCh poles in three
  //     shared-memory buffers: while warp 0 decides chunk ch (rotate or keep, FP64
  //     work only after a rotation that the speculation did not cover) and assigns
  //     its records, the other warps write the records of chunk ch-1 and stage the
  //     inputs of chunk ch+1.
  constexpr int kCh = 128;
  __shared__ int sc_c[3][kCh];
  __shared__ uint8_t sc_f[3][kCh], o_code[3][kCh];
  __shared__ int o_idx[3][kCh], o_cidx[3][kCh], o_pj[3][kCh], o_sup[3][kCh];
  __shared__ double sc_D[3][kCh], sc_z[3][kCh], sc_cs[3][kCh], sc_sn[3][kCh], sc_tau[3][kCh], sc_dp[3][kCh],
      sc_di[3][kCh];
  auto stage = [&](int b, int q0, int t0, int nt) {
    for (int i = t0; i < kCh; i += nt) {
      const int q = q0 + i;
      if (q >= nL) break;
      const int c = V.perm[v0 + Lpos[q]];
      sc_c[b][i] = c;
      sc_D[b][i] = V.Dc[v0 + c];
      sc_z[b][i] = V.zc[v0 + c];
      const uint8_t f = q > 0 ? flag[q] : 0;
      sc_f[b][i] = f;
      if (f & 1) {
        sc_cs[b][i] = spc[q];
        sc_sn[b][i] = spc[n + q];
        sc_tau[b][i] = stau[q];
        sc_dp[b][i] = sdp[q];
        sc_di[b][i] = sdi[q];
      }
    }
  };
  // records of a decided chunk: code bit 0 = rotation (else the previous survivor
  // is kept), bit 1 = first rotation of a chain; values in sc_cs/sc_sn/sc_dp
  // (rotation: c, s, deflated value) or sc_cs/sc_sn (kept: pole, weight)
  auto emit = [&](int b, int q0, int t0, int nt) {
    for (int i = t0; i < kCh; i += nt) {
      const int q = q0 + i;
      if (q >= nL) break;
      if (q == 0) continue;
      const uint8_t code = o_code[b][i];
      const int idx = o_idx[b][i], pjq = o_pj[b][i], sup = o_sup[b][i];
      if (code & 1) {
        const int64_t ro = v0 + idx;
        V.rij[4 * ro + 0] = pjq;
        V.rij[4 * ro + 1] = sc_c[b][i];
        V.rij[4 * ro + 2] = sup;
        V.rcs[2 * ro + 0] = sc_cs[b][i];
        V.rcs[2 * ro + 1] = sc_sn[b][i];
        if (code & 2) V.rch[v0 + o_cidx[b][i]] = idx;
        const int d = t1 + idx;
        V.dcol[v0 + d] = pjq;
        V.dval[v0 + d] = sc_dp[b][i];
        V.dseg[v0 + d] = (uint8_t)((sup & 0xff) | (sup >> 8));
      } else {
        V.kept[v0 + idx] = pjq;
        V.Dk[v0 + idx] = sc_cs[b][i];
        V.zk[v0 + idx] = sc_sn[b][i];
        V.kseg[v0 + idx] = (uint8_t)sup;
      }
    }
  };
  const int nch_chunks = (nL + kCh - 1) / kCh;
  stage(0, 0, threadIdx.x, blockDim.x);
  __syncthreads();
  // warp 0 decides, 32 poles at a time.  Its lanes run, in step, the scan's state
  // machine over the sub-chunk's speculative bits: N (the candidate is an original pole: the pair's
  // test is bit 0), S (the candidate came from a bit-0 rotation: bit 1), X (it came from
  // any other rotation: the test and the rotation in FP64, the only sequential FP64
  // work); it jumps over runs of N without a bit-0 rotation.  Each lane then derives its
  // pole's record from the decision word: indices from popcounts, the candidate (the
  // previous pole, its values those left by a rotation at it), the candidate's support
  // as the OR of the supports along the run of rotations that built it.
  int K = 0, nr = 0, nch = 0;
  int st = 0, cpj = -1, cps = 0;  // scan state and the candidate after the last decided pole
  double cpD = 0.0, cpz = 0.0;
  bool cprot = false;             // the last decided pole rotated
  for (int ch = 0; ch < nch_chunks; ++ch) {
    const int b = ch % 3;
    if (threadIdx.x >= 32) {
      if (ch > 0) emit((ch + 2) % 3, (ch - 1) * kCh, threadIdx.x - 32, blockDim.x - 32);
      stage((ch + 1) % 3, (ch + 1) * kCh, threadIdx.x - 32, blockDim.x - 32);
    }
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      const int qend = min(kCh, nL - ch * kCh);
      for (int s0 = 0; s0 < qend; s0 += 32) {
        const int i = s0 + lane, q = ch * kCh + i;
        const bool valid = i < qend;
        const uint8_t f = valid ? sc_f[b][i] : 0;
        const int cq = valid ? sc_c[b][i] : 0;
        const int spq = cq < n1 ? 1 : 2;
        const unsigned vm = __ballot_sync(0xffffffffu, valid);
        const unsigned b0 = __ballot_sync(0xffffffffu, valid && q > 0 && (f & 1));
        const unsigned b1 = __ballot_sync(0xffffffffu, valid && q > 0 && (f & 2));
        const unsigned topm = __ballot_sync(0xffffffffu, valid && spq == 1);
        const unsigned botm = __ballot_sync(0xffffffffu, valid && spq == 2);
        const int kn = min(32, qend - s0);
        unsigned rotw = 0;
        int sn = st;
        // no bit-0 rotation right after a rotation and no S pole with bit 1: the
        // decisions are the bit-0 word itself (isolated pairs of equal poles)
        const unsigned kmask = kn >= 32 ? 0xffffffffu : ((1u << kn) - 1u);
        const unsigned sS = (b0 << 1) | (st == 1 ? 1u : 0u);
        if (st != 2 && (b0 & sS) == 0u && (b1 & sS & kmask) == 0u) {
          rotw = b0;
          sn = ((b0 >> (kn - 1)) & 1u) ? 1 : 0;
        } else {  // every lane runs it on the same warp-uniform words: uniform branches
          int k = 0;
          while (k < kn) {
            if (ch * kCh + s0 + k == 0) {
              sn = 0;
              ++k;
              continue;
            }
            if (sn == 0) {
              const unsigned m = b0 >> k;
              if (m == 0u) break;
              k += __ffs(m) - 1;
              rotw |= 1u << k;
              sn = 1;
              ++k;
              continue;
            }
            if (sn == 1 && ((b1 >> k) & 1u) == 0u) {  // the rotated survivor is kept: bits only
              sn = 0;
              ++k;
              continue;
            }
            // a rotation after a rotation: bit 1 (S) says so, X tests in FP64
            const int ii = s0 + k;
            const double Dq = sc_D[b][ii], zq = sc_z[b][ii];
            const double pDv = k > 0 ? sc_di[b][ii - 1] : cpD, pzv = k > 0 ? sc_tau[b][ii - 1] : cpz;
            bool r = true;
            if (sn == 2) r = type2_test(Dq, zq, pDv, pzv, tol);
            if (r) {
              double cc, ss, tau, dp, di;
              type2_rot(Dq, zq, pDv, pzv, cc, ss, tau, dp, di);
              __syncwarp();  // every lane has read the candidate before lane 0 writes
              if (lane == 0) {
                sc_cs[b][ii] = cc;
                sc_sn[b][ii] = ss;
                sc_dp[b][ii] = dp;
                sc_tau[b][ii] = tau;
                sc_di[b][ii] = di;
              }
              __syncwarp();
              rotw |= 1u << k;
              sn = 2;
            } else {
              sn = 0;
            }
            ++k;
          }
        }
        __syncwarp();
        const unsigned prevw = (rotw << 1) | (cprot ? 1u : 0u);
        const unsigned starts = rotw & ~prevw;
        const unsigned keepw = ~rotw & vm & ((ch == 0 && s0 == 0) ? ~1u : ~0u);
        // OR of the supports over the run of rotations ending at sub-chunk index m
        auto run_sup = [&](int m) -> int {
          const unsigned upto = m >= 31 ? 0xffffffffu : ((2u << m) - 1u);
          const unsigned zeros = ~rotw & upto & vm;
          unsigned range = upto;
          int extra = cps;
          if (zeros) {
            range = upto & ~((1u << (31 - __clz(zeros))) - 1u);
            extra = 0;
          }
          return extra | ((topm & range) ? 1 : 0) | ((botm & range) ? 2 : 0);
        };
        if (valid && q > 0) {
          const unsigned lt = (1u << lane) - 1u;
          const bool rot = ((rotw >> lane) & 1u) != 0u, prot = ((prevw >> lane) & 1u) != 0u;
          const int ps = lane > 0 ? run_sup(lane - 1) : cps;
          o_pj[b][i] = lane > 0 ? sc_c[b][i - 1] : cpj;
          if (rot) {
            o_code[b][i] = prot ? 1 : 3;
            o_idx[b][i] = nr + __popc(rotw & lt);
            if (!prot) o_cidx[b][i] = nch + __popc(starts & lt);
            o_sup[b][i] = ps | (spq << 8);
          } else {
            o_code[b][i] = 0;
            o_idx[b][i] = K + __popc(keepw & lt);
            o_sup[b][i] = ps;
            sc_cs[b][i] = lane == 0 ? cpD : (prot ? sc_di[b][i - 1] : sc_D[b][i - 1]);
            sc_sn[b][i] = lane == 0 ? cpz : (prot ? sc_tau[b][i - 1] : sc_z[b][i - 1]);
          }
        }
        const int last = kn - 1;
        const bool lr = ((rotw >> last) & 1u) != 0u;
        const int nps = run_sup(last);
        cpj = __shfl_sync(0xffffffffu, cq, last);
        cpD = lr ? sc_di[b][s0 + last] : sc_D[b][s0 + last];
        cpz = lr ? sc_tau[b][s0 + last] : sc_z[b][s0 + last];
        cps = nps;
        cprot = lr;
        st = sn;
        K += __popc(keepw);
        nr += __popc(rotw);
        nch += __popc(starts);
        __syncwarp();
      }
    }
    __syncthreads();
  }
  if (nch_chunks > 0) emit((nch_chunks - 1) % 3, (nch_chunks - 1) * kCh, threadIdx.x, blockDim.x);
  const int ndf = t1 + nr;
  if (threadIdx.x == 0) {
    if (cpj >= 0) {
      V.kept[v0 + K] = cpj; V.Dk[v0 + K] = cpD; V.zk[v0 + K] = cpz; V.kseg[v0 + K] = (uint8_t)cps; ++K;
    }
    sres[0] = K; sres[1] = ndf; sres[2] = nr; sres[3] = nch;
    P.m.K[g] = K; P.m.nd[g] = ndf; P.m.nrot[g] = nr; P.m.nchain[g] = nch;
    if (P.stats && level < TDC_MAX_LEVELS) {
      atomicAdd(&P.stats->sum_n[level], (unsigned long long)n);
      atomicAdd(&P.stats->sum_K[level], (unsigned long long)K);
      atomicAdd(&P.stats->n_rot[level], (unsigned long long)nr);
      atomicAdd(&P.stats->n_type1[level], (unsigned long long)t1);
      atomicAdd(&P.stats->n_merges[level], 1ull);
      atomicMax(&P.stats->max_K[level], K);
    }
  }
  __syncthreads();
  const int Kf = sres[0];
  // 4. lists of non-deflated poles with support in the top / bottom rows
  const int perk = (Kf + blockDim.x - 1) / blockDim.x;
  const int j0 = min(Kf, (int)threadIdx.x * perk), j1 = min(Kf, j0 + perk);
  int ct = 0, cb = 0;
  for (int j = j0; j < j1; ++j) {
    uint8_t s = V.kseg[v0 + j];
    ct += (s & 1) ? 1 : 0;
    cb += (s & 2) ? 1 : 0;
  }
  int ot = ct, ob = cb;
  block_excl_scan2(ot, ob, redi);
  for (int j = j0; j < j1; ++j) {
    uint8_t s = V.kseg[v0 + j];
    if (s & 1) V.tlist[v0 + ot++] = j;
    if (s & 2) V.blist[v0 + ob++] = j;
  }
  // FP32 copies for the secular pre-iteration: coordinate relative to a centre pole
  // (as an unevaluated sum of two floats, xz.x + xlo) and the squared weight
  if (Kf > 0) {
    const double dc = V.Dk[v0 + (Kf >> 1)];
    for (int j = threadIdx.x; j < Kf; j += blockDim.x) {
      const double zj = V.zk[v0 + j];
      const double x = V.Dk[v0 + j] - dc;
      const float xh = (float)x;
      V.xz[v0 + j] = make_float2(xh, (float)(zj * zj));
      V.zz[v0 + j] = zj * zj;
      V.xlo[v0 + j] = (float)(x - (double)xh);
    }
  }
  if (threadIdx.x == blockDim.x - 1) {
    P.m.ntop[g] = ot;
    P.m.nbot[g] = ob;
    if (P.stats && level < TDC_MAX_LEVELS)
      atomicAdd(&P.stats->gemm_flops[level],
                2ull * ((unsigned long long)n1 * ot + (unsigned long long)(n - n1) * ob) * (unsigned long long)Kf);
  }
}

cudaError_t launch_prepare(const Plan& P, const LevelLaunch& L, cudaStream_t s) {
  int threads = 256;
  while (threads > 64 && threads / 2 >= L.max_n) threads /= 2;
  // a level of fewer merges than SMs: a wider block per merge (down to 16 poles a thread)
  // shortens the level's critical path; the outputs do not depend on the block size
  if (L.merges < 152)
    while (threads < 1024 && (int64_t)threads * 16 <= L.max_n) threads *= 2;
  k_prepare<<<(unsigned)L.merges, threads, 0, s>>>(P, L.level);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// k_rotate: apply the deflation rotations to Q's columns.  Rows are
// independent; chains of rotations that share a column run in order; distinct
// chains touch disjoint columns.  An entry outside a column's row support
// (top or bottom child) is a structural zero and is never read.
// ---------------------------------------------------------------------------
static constexpr int kRotChainsPerGrid = 512;

__global__ void __launch_bounds__(256) k_rotate(Plan P, int level) {
  const int64_t g = blockIdx.x;
  const int nr = P.m.nrot[g];
  if (nr == 0) return;
  const Node nd = make_node(P, level, g);
  const int n = (int)(nd.hi - nd.lo), n1 = (int)(nd.mid - nd.lo);
  const int r = blockIdx.y * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int half = r < n1 ? 1 : 2;
  const int nch = P.m.nchain[g];
  const int64_t v0 = nd.v0;
  double* col = nd.src + r;
  for (int h = blockIdx.z; h < nch; h += gridDim.z) {
    const int k0 = P.v.rch[v0 + h];
    const int k1 = (h + 1 < nch) ? P.v.rch[v0 + h + 1] : nr;
    for (int k = k0; k < k1; ++k) {
      const int pj = P.v.rij[4 * (v0 + k) + 0];
      const int ci = P.v.rij[4 * (v0 + k) + 1];
      const int sup = P.v.rij[4 * (v0 + k) + 2];
      const int sp = sup & 0xff, si = sup >> 8;
      if (!((sp | si) & half)) continue;
      const double c = P.v.rcs[2 * (v0 + k)], s = P.v.rcs[2 * (v0 + k) + 1];
      const double x = (sp & half) ? col[(int64_t)pj * nd.lds] : 0.0;
      const double y = (si & half) ? col[(int64_t)ci * nd.lds] : 0.0;
      col[(int64_t)pj * nd.lds] = c * x + s * y;
      col[(int64_t)ci * nd.lds] = c * y - s * x;
    }
  }
}

cudaError_t launch_rotate(const Plan& P, const LevelLaunch& L, cudaStream_t s) {
  // chains are spread over grid.z; small merges (many per level) need few
  const unsigned gz = (unsigned)std::max<int64_t>(1, std::min<int64_t>(kRotChainsPerGrid, L.max_n / 32));
  dim3 grid((unsigned)L.merges, (unsigned)((L.max_n + 255) / 256), gz);
  k_rotate<<<grid, 256, 0, s>>>(P, L.level);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Root-slot mapping: warp w of the level handles vector slot w.
// ---------------------------------------------------------------------------
struct Slot {
  bool valid;
  int64_t g;      // merge index on the level
  int j;          // root / pole index within the merge
  int K;
  int64_t v0;
  double rho;
};

__device__ __forceinline__ Slot slot_of(const Plan& P, int level, int nprob_act, int64_t s) {
  Slot o;
  o.valid = false;
  int pi = find_problem_by_slot(P.prob, nprob_act, s);
  const Problem& p = P.prob[pi];
  int64_t r = s - p.voff;
  if (r < 0 || r >= p.n) return o;
  int64_t i = node_of_row(r, p.n, level);
  int64_t lo = node_bound(i, p.n, level);
  int64_t mid = node_bound(2 * i + 1, p.n, level + 1);
  o.g = ((int64_t)pi << level) + i;
  o.j = (int)(r - lo);
  o.K = P.m.K[o.g];
  o.v0 = p.voff + lo;
  o.rho = 2.0 * fabs(input_entry(P.e[p.off_de + mid - 1], p.escale));
  o.valid = o.j < o.K;
  return o;
}

// ---------------------------------------------------------------------------
// k_secular: root j of 1/rho + sum_i z_i^2/(d_i - lambda) = 0 (Eq. (secular)).
// Origin: d_j when the function is >= 0 at the midpoint of (d_j, d_{j+1}),
// else d_{j+1}; the last root is measured from d_{K-1}.  With
// delta_i = d_i - d_org, g(tau) = 1/rho + sum_i z_i^2/(delta_i - tau).
// Iteration: the two sums over poles left (psi) and right (phi) of the root
// are each replaced by a constant plus one pole term matching value and slope
// at tau (the nearest poles d_j, d_{j+1}); the model's root is the next iterate
// (a quadratic), safeguarded by bisection on the bracket.
// ---------------------------------------------------------------------------
// W = 32: the warp's lanes share the poles and the sums are reduced over the
// warp; W = 1: one thread takes every pole (small merges, a root per thread).
template <int W = 32>
__device__ __forceinline__ void secular_sums(const double* D, const double* z, int K, int j, double dorg,
                                             double tau, double& psi, double& dpsi, double& phi,
                                             double& dphi, double& sabs) {
  const int lane = W == 32 ? (threadIdx.x & 31) : 0;
  double a = 0.0, da = 0.0, b = 0.0, db = 0.0;
  // poles left of the root (i <= j) give negative terms, poles right of it positive
  // ones, so sum |t| = phi - psi needs no separate accumulation
  const int split = min(K, j + 1);
  for (int i = lane; i < split; i += W) {
    const double r = rcp_nr((D[i] - dorg) - tau);
    const double zi = z[i];
    const double t = zi * zi * r;
    a += t;
    da = fma(t, r, da);
  }
  for (int i = split + lane; i < K; i += W) {
    const double r = rcp_nr((D[i] - dorg) - tau);
    const double zi = z[i];
    const double t = zi * zi * r;
    b += t;
    db = fma(t, r, db);
  }
  if (W == 32) {
    a = warp_sum(a);
    da = warp_sum(da);
    b = warp_sum(b);
    db = warp_sum(db);
  }
  psi = a;
  dpsi = da;
  phi = b;
  dphi = db;
  sabs = phi - psi;
}

// Next iterate from the two-pole rational model of g at tau: psi and phi are
// each replaced by a constant plus the term of the nearest pole on their side
// (d_j at dl, d_{j+1} at dr, in the origin's frame), matching value and slope;
// the model's root in the bracket (lo, hi), else the bracket's midpoint.
__device__ __forceinline__ double model_step(int j, int K, double irho, double dl, double dr, double tau, double gv,
                                             double psi, double dpsi, double phi, double dphi, double lo,
                                             double hi) {
  const double p = dl - tau;  // < 0
  double h = 0.0;
  bool ok = true;
  if (j < K - 1) {
    const double q = dr - tau;  // > 0
    const double b1 = dpsi * p * p, b2 = dphi * q * q;
    const double A = irho + (psi - b1 / p) + (phi - b2 / q);
    const double B = A * (p + q) + b1 + b2;
    const double C = p * q * gv;
    if (A == 0.0) {
      h = C / B;
    } else {
      const double disc = B * B - 4.0 * A * C;
      if (disc < 0.0) {
        ok = false;
      } else {
        const double w = B + copysign(sqrt(disc), B);
        const double h1 = (w != 0.0) ? 2.0 * C / w : 0.0;
        const double h2 = w / (2.0 * A);
        const bool in1 = (h1 > p && h1 < q), in2 = (h2 > p && h2 < q);
        if (in1 && (!in2 || fabs(h1) <= fabs(h2))) h = h1;
        else if (in2) h = h2;
        else ok = false;
      }
    }
  } else {
    const double b1 = dpsi * p * p;
    const double A = irho + (psi - b1 / p) + phi;
    if (A != 0.0) h = p + b1 / A; else ok = false;
  }
  double tn = tau + h;
  if (!ok || !(tn > lo && tn < hi) || !isfinite(tn)) tn = 0.5 * (lo + hi);
  return tn;
}

// FP64 iteration for root j from origin org, starting at tau inside [lo, hi] with
// the sums at tau already known.  Two-pole rational model of g around tau (the
// nearest poles exact), safeguarded by bisection; stops when |g| is at rounding
// level of 1/rho + sum |t| or the step is below rounding level of tau.  Returns
// the number of passes over the poles (sum evaluations) made.
template <int W = 32>
__device__ int secular_fp64(const double* D, const double* z, int K, int j, double irho, int org, double& tau,
                            double& lo, double& hi, double psi, double dpsi, double phi, double dphi, double sabs,
                            int max_iter, bool& conv) {
  const double dorg = D[org];
  const double dl = D[j] - dorg;                         // delta_j (0 when org == j)
  const double dr = (j < K - 1) ? D[j + 1] - dorg : 0.0; // delta_{j+1}
  int passes = 0;
  conv = false;
  for (int it = 1; it <= max_iter; ++it) {
    if (it > 1) {
      secular_sums<W>(D, z, K, j, dorg, tau, psi, dpsi, phi, dphi, sabs);
      ++passes;
    }
    const double gv = irho + psi + phi;
    if (gv == 0.0 || fabs(gv) <= 8.0 * kEps * (irho + sabs)) { conv = true; break; }
    if (gv < 0.0) lo = tau; else hi = tau;
    const double tn = model_step(j, K, irho, dl, dr, tau, gv, psi, dpsi, phi, dphi, lo, hi);
    const bool small_step = fabs(tn - tau) <= 2.0 * kEps * fabs(tau);
    tau = tn;
    if (small_step || (hi - lo) <= 2.0 * kEps * fmax(fabs(lo), fabs(hi))) { conv = true; break; }
  }
  return passes;
}

// FP64 iteration for root j from a close starting point (the FP32 estimate)
// with a single pass over all poles.  In that pass, at tau1, the term of each
// lane's pole in the window [j-15, j+16] (the 32 poles nearest the root) is kept
// apart from the far terms, whose sums of t, t r and t r^2 (r = 1/(delta_i - tau1))
// are kept per side.  The following iterates tau = tau1 + e re-evaluate only the
// window terms; the far sums follow from
//   t_i(tau1 + e) = t_i / (1 - e r_i) = t_i (1 + e r_i + (e r_i)^2) + rest_i,
//   |sum of rest_i| <= (sum of far |t_i|) q^3 / (1 - q),  q = |e| / (distance from
//   tau1 to the nearest far pole),
// (their slopes likewise, to first order, for the model only).  A root is
// accepted when |g| plus that bound passes the convergence test.  Returns true
// when accepted (tau updated, conv set); otherwise tau is the last iterate,
// lo / hi hold the bracket, and the caller continues with full passes.
__device__ bool secular_certified(const double* D, const double* z, const double* zz, int K, int j, double irho,
                                  int org, double& tau, double& lo, double& hi, bool& conv) {
  const int lane = threadIdx.x & 31;
  const double dorg = D[org];
  const double dl = D[j] - dorg, dr = (j < K - 1) ? D[j + 1] - dorg : 0.0;
  const int wlo = j - 15, whi = j + 16;
  const int iw = wlo + ((lane - wlo) & 31);  // this lane's window pole
  const bool wv = iw >= 0 && iw < K, wleft = iw <= j;
  const double zw2 = wv ? zz[iw] : 0.0, dw = wv ? D[iw] - dorg : 0.0;
  const double tau1 = tau;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, b0 = 0.0, b1 = 0.0, b2 = 0.0, wt = 0.0, wd = 0.0;
  // this lane's poles are i = lane (mod 32): those below the window lie left of the
  // root, its one window pole iw is kept apart, those above the window lie right
  // of it -- three branch-free ranges
  for (int i = lane; i < wlo; i += 32) {
    const double r = rcp_nr((D[i] - dorg) - tau1);
    const double t = zz[i] * r, tr = t * r;
    a0 += t; a1 += tr; a2 = fma(tr, r, a2);
  }
  if (wv) {
    const double r = rcp_nr(dw - tau1);
    wt = zw2 * r;
    wd = wt * r;
  }
  for (int i = iw + 32; i < K; i += 32) {
    const double r = rcp_nr((D[i] - dorg) - tau1);
    const double t = zz[i] * r, tr = t * r;
    b0 += t; b1 += tr; b2 = fma(tr, r, b2);
  }
  a0 = warp_sum(a0); a1 = warp_sum(a1); a2 = warp_sum(a2);
  b0 = warp_sum(b0); b1 = warp_sum(b1); b2 = warp_sum(b2);
  // distance from tau1 to the nearest far pole (poles are sorted)
  double dmin = HUGE_VAL;
  if (wlo - 1 >= 0) dmin = fmin(dmin, fabs((D[wlo - 1] - dorg) - tau1));
  if (whi + 1 < K) dmin = fmin(dmin, fabs((D[whi + 1] - dorg) - tau1));
  conv = false;
  double tc = tau1;
  for (int k = 0; k < 8; ++k) {
    const double e = tc - tau1;
    const double q = fabs(e) / dmin;
    // beyond q ~ eps^(1/3) the expansion is no better than a full evaluation
    if (!(q < 4e-6)) break;
    if (k > 0) {  // window terms at tc
      wt = 0.0;
      wd = 0.0;
      if (wv) {
        const double r = rcp_nr(dw - tc);
        wt = zw2 * r;
        wd = wt * r;
      }
    }
    const double wtl = warp_sum((wv && wleft) ? wt : 0.0), wtr = warp_sum((wv && !wleft) ? wt : 0.0);
    const double wdl = warp_sum((wv && wleft) ? wd : 0.0), wdr = warp_sum((wv && !wleft) ? wd : 0.0);
    const double rest = k > 0 ? (b0 - a0) * (q * q * q) / (1.0 - q) : 0.0;
    const double psi = a0 + e * (a1 + e * a2) + wtl, dpsi = a1 + 2.0 * e * a2 + wdl;
    const double phi = b0 + e * (b1 + e * b2) + wtr, dphi = b1 + 2.0 * e * b2 + wdr;
    const double gv = irho + psi + phi;
    if (gv == 0.0 || fabs(gv) + rest <= 8.0 * kEps * (irho + (phi - psi))) {
      tau = tc;
      conv = true;
      return true;
    }
    if (fabs(gv) > rest) {
      if (gv < 0.0) lo = tc; else hi = tc;
    }
    const double tn = model_step(j, K, irho, dl, dr, tc, gv, psi, dpsi, phi, dphi, lo, hi);
    // a vanishing step counts only where g is known to rounding level
    const bool exact_g = rest <= kEps * (irho + (phi - psi));
    if (exact_g && (fabs(tn - tc) <= 2.0 * kEps * fabs(tc) || (hi - lo) <= 2.0 * kEps * fmax(fabs(lo), fabs(hi)))) {
      tau = tn;
      conv = true;
      return true;
    }
    tc = tn;
  }
  tau = tc;
  return false;
}

// FP32 pre-iteration for root j: width = d_{j+1} - d_j, or for the last root
// width = rho |z|^2.  Far poles use the two-float coordinates (xz[i].x + xlo[i] =
// d_i - d_c, one centre per merge) and xz[i].y = z_i^2; the 32 poles nearest to j
// (one per lane) use their FP64 differences.  The first evaluation, at the middle
// of the interval, picks the frame: tau is kept relative to the nearer pole o (j,
// or j+1 with tau < 0), so a root close to d_j+1 keeps its relative precision.
// Interior roots start at the midpoint with the two-pole model; the last root
// starts from the root of g with every other pole frozen at tau = 0 (it often
// lies far below the interval's middle) and iterates the one-pole model.
// Returns false if no usable estimate; otherwise org_out and tau_out.
__device__ bool secular_fp32(const double* D, const float2* xz, const float* xlo, int K, int j, float irho,
                             float width, int& org_out, float& tau_out) {
  const int lane = threadIdx.x & 31;
  const bool last = j == K - 1;
  // the window pole of this lane: the i = lane (mod 32) in [j - 15, j + 16]
  const int iw = j - 15 + ((lane - (j - 15)) & 31);
  const bool wv = iw >= 0 && iw < K;
  float dw = wv ? (float)(D[iw] - D[j]) : 0.0f;
  int o = j;
  float xo = xz[j].x, xlo_o = xlo[j];
  float lo = 0.0f, hi = width, tau = 0.5f * width;
  for (int it = 0; it < 12; ++it) {
    // it == 0 for the last root: the sum of the other poles' terms at tau = 0
    const float tv = (last && it == 0) ? 0.0f : tau;
    float a = 0.0f, da = 0.0f, b = 0.0f, db = 0.0f;
    for (int i = lane; i < K; i += 32) {
      const float2 v = xz[i];
      const float del = (i == iw) ? dw : (v.x - xo) + (xlo[i] - xlo_o);
      if (last && it == 0 && i == j) continue;
      float r;
      asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(del - tv));
      const float t = v.y * r;
      if (i <= j) { a += t; da = fmaf(t, r, da); }
      else { b += t; db = fmaf(t, r, db); }
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, s);
      da += __shfl_xor_sync(0xffffffffu, da, s);
      b += __shfl_xor_sync(0xffffffffu, b, s);
      db += __shfl_xor_sync(0xffffffffu, db, s);
    }
    if (last && it == 0) {
      const float den = irho + a;
      const float t0 = den > 0.0f ? xz[j].y / den : -1.0f;
      if (t0 > 0.0f && t0 < width) tau = t0;
      continue;
    }
    const float gv = irho + a + b;
    if (!isfinite(gv)) return false;
    if (gv == 0.0f) break;
    if (it == 0 && !last && gv < 0.0f) {
      // root in the upper half: continue in the frame of pole j+1 (same point)
      o = j + 1;
      xo = xz[j + 1].x;
      xlo_o = xlo[j + 1];
      dw = wv ? (float)(D[iw] - D[j + 1]) : 0.0f;
      tau = -0.5f * width;
      lo = -width;
      hi = 0.0f;
    }
    if (gv < 0.0f) lo = tau; else hi = tau;
    // p = d_j - lambda, q = d_j+1 - lambda in the current frame
    const float p = o == j ? -tau : -(width + tau);
    float h = 0.0f;
    bool ok = true;
    if (last) {
      const float b1 = da * p * p;
      const float A = irho + (a - b1 / p) + b;
      if (A != 0.0f) h = p + b1 / A; else ok = false;
    } else {
      const float q = o == j ? width - tau : -tau;
      const float b1 = da * p * p, b2 = db * q * q;
      const float A = irho + (a - b1 / p) + (b - b2 / q);
      const float B = A * (p + q) + b1 + b2;
      const float C = p * q * gv;
      if (A == 0.0f) {
        h = C / B;
      } else {
        const float disc = B * B - 4.0f * A * C;
        if (disc < 0.0f) {
          ok = false;
        } else {
          const float w = B + copysignf(sqrtf(disc), B);
          const float h1 = (w != 0.0f) ? 2.0f * C / w : 0.0f;
          const float h2 = w / (2.0f * A);
          const bool in1 = (h1 > p && h1 < q), in2 = (h2 > p && h2 < q);
          if (in1 && (!in2 || fabsf(h1) <= fabsf(h2))) h = h1;
          else if (in2) h = h2;
          else ok = false;
        }
      }
    }
    float tn = tau + h;
    if (!ok || !(tn > lo && tn < hi) || !isfinite(tn)) tn = 0.5f * (lo + hi);
    const bool small = fabsf(tn - tau) <= 2e-7f * fabsf(tau);
    tau = tn;
    if (small || (hi - lo) <= 4e-7f * fmaxf(fabsf(lo), fabsf(hi))) break;
  }
  if (o == j ? !(tau > 0.0f && tau < width) : !(tau > -width && tau < 0.0f)) return false;
  org_out = o;
  tau_out = tau;
  return true;
}

// Warp-cooperative solve of root j; every lane returns the same (org, tau).
// With xz (FP32 copies of the poles and weights) the root is first located in
// FP32; its position picks the origin (the nearer pole) and the FP64 iteration
// starts there, with the whole interval as bracket.  A root that converges in
// the half of the far pole is re-solved from that pole.  Without xz, or when the
// FP32 estimate is unusable, the origin comes from the sign of g at the midpoint.
__device__ void secular_root(const double* D, const double* z, const double* zz, const float2* xz, const float* xlo,
                             int K, int j,
                             double rho, int max_iter, int& org_out, double& tau_out, int& iters, bool& conv) {
  const double irho = 1.0 / rho;
  int org;
  double lo, hi, tau;
  double psi, dpsi, phi, dphi, sabs;
  int passes = 1;
  const bool last = j == K - 1;
  double width;
  if (!last) {
    width = D[j + 1] - D[j];
  } else {
    double zz = 0.0;
    for (int i = threadIdx.x & 31; i < K; i += 32) zz = fma(z[i], z[i], zz);
    width = rho * warp_sum(zz);
  }
  float t32 = 0.0f;
  int o32 = j;
  if (xz != nullptr && width > 0.0 && secular_fp32(D, xz, xlo, K, j, (float)irho, (float)width, o32, t32)) {
    org = o32;
    tau = (double)t32;
    if (org == j) { lo = 0.0; hi = width; } else { lo = -width; hi = 0.0; }
    if (!(tau > lo && tau < hi)) tau = 0.5 * (lo + hi);
    const bool tried = max_iter >= 2;
    if (!tried || !secular_certified(D, z, zz, K, j, irho, org, tau, lo, hi, conv)) {
      secular_sums(D, z, K, j, D[org], tau, psi, dpsi, phi, dphi, sabs);
      if (tried) ++passes;
      passes += secular_fp64(D, z, K, j, irho, org, tau, lo, hi, psi, dpsi, phi, dphi, sabs, max_iter, conv);
    }
    // an interior root that converged nearer the other pole: continue from that pole
    const bool far = !last && conv && ((org == j) ? (tau > 0.5 * width) : (tau < -0.5 * width));
    if (far) {
      if (org == j) { org = j + 1; tau -= width; lo -= width; hi -= width; }
      else { org = j; tau += width; lo += width; hi += width; }
      secular_sums(D, z, K, j, D[org], tau, psi, dpsi, phi, dphi, sabs);
      ++passes;
      passes += secular_fp64(D, z, K, j, irho, org, tau, lo, hi, psi, dpsi, phi, dphi, sabs, max_iter, conv);
    }
    org_out = org;
    tau_out = tau;
    iters = min(passes, max_iter);
    return;
  }
  if (!last) {
    secular_sums(D, z, K, j, D[j], 0.5 * width, psi, dpsi, phi, dphi, sabs);
    if (irho + psi + phi >= 0.0) { org = j; lo = 0.0; hi = 0.5 * width; tau = hi; }
    else { org = j + 1; lo = -0.5 * width; hi = 0.0; tau = lo; }
  } else {
    org = K - 1; lo = 0.0; hi = width; tau = hi;
    secular_sums(D, z, K, j, D[org], tau, psi, dpsi, phi, dphi, sabs);
  }
  passes += secular_fp64(D, z, K, j, irho, org, tau, lo, hi, psi, dpsi, phi, dphi, sabs, max_iter, conv);
  org_out = org;
  tau_out = tau;
  iters = min(passes, max_iter);
}

// FP32 pre-iteration of one thread for root j of a small merge.  Pole differences
// come from the two-float coordinates, (x_i - x_o) + (xlo_i - xlo_o), accurate to
// a few FP32 roundings of d_i - d_o itself however far the poles lie from the
// merge's centre.  The first evaluation, at the middle of (d_j, d_j+1), picks the
// frame: tau is kept relative to the nearer pole o (j, or j+1 with tau < 0), so a
// root close to d_j+1 keeps its relative precision instead of rounding onto
// width.  The model steps are those of the warp version (two-pole for interior
// roots from the midpoint; one-pole for the last root from its frozen-poles
// start).  Returns false if no usable estimate; otherwise org_out and tau_out.
__device__ bool secular_fp32_thread(const float2* xz, const float* xlo, int K, int j, float irho, float width,
                                    int& org_out, float& tau_out) {
  const bool last = j == K - 1;
  int o = j;
  float xo = xz[j].x, xlo_o = xlo[j];
  float lo = 0.0f, hi = width, tau = 0.5f * width;
  for (int it = 0; it < 12; ++it) {
    const float tv = (last && it == 0) ? 0.0f : tau;
    float a = 0.0f, da = 0.0f, b = 0.0f, db = 0.0f;
    // poles left of the root and right of it in two loops (each lane its own j):
    // no divergent branch inside the loop
    auto term = [&](int i, float& acc, float& dacc) {
      const float2 v = xz[i];
      const float del = (v.x - xo) + (xlo[i] - xlo_o);
      float r;
      asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(del - tv));
      const float t = v.y * r;
      acc += t;
      dacc = fmaf(t, r, dacc);
    };
    const int jl = (last && it == 0) ? j : j + 1;  // the last root's first pass leaves out pole j
    for (int i = 0; i < jl; ++i) term(i, a, da);
    for (int i = j + 1; i < K; ++i) term(i, b, db);
    if (last && it == 0) {
      const float den = irho + a;
      const float t0 = den > 0.0f ? xz[j].y / den : -1.0f;
      if (t0 > 0.0f && t0 < width) tau = t0;
      continue;
    }
    const float gv = irho + a + b;
    if (!isfinite(gv)) return false;
    if (gv == 0.0f) break;
    if (it == 0 && !last && gv < 0.0f) {
      // root in the upper half: continue in the frame of pole j+1 (same point)
      o = j + 1;
      xo = xz[j + 1].x;
      xlo_o = xlo[j + 1];
      tau = -0.5f * width;
      lo = -width;
      hi = 0.0f;
    }
    if (gv < 0.0f) lo = tau; else hi = tau;
    // p = d_j - lambda, q2 = d_j+1 - lambda in the current frame
    const float p = o == j ? -tau : -(width + tau);
    float h = 0.0f;
    bool ok = true;
    if (last) {
      const float b1 = da * p * p;
      const float A = irho + (a - b1 / p) + b;
      if (A != 0.0f) h = p + b1 / A; else ok = false;
    } else {
      const float q2 = o == j ? width - tau : -tau;
      const float b1 = da * p * p, b2 = db * q2 * q2;
      const float A = irho + (a - b1 / p) + (b - b2 / q2);
      const float B = A * (p + q2) + b1 + b2;
      const float C = p * q2 * gv;
      if (A == 0.0f) {
        h = C / B;
      } else {
        const float disc = B * B - 4.0f * A * C;
        if (disc < 0.0f) {
          ok = false;
        } else {
          const float w = B + copysignf(sqrtf(disc), B);
          const float h1 = (w != 0.0f) ? 2.0f * C / w : 0.0f;
          const float h2 = w / (2.0f * A);
          const bool in1 = (h1 > p && h1 < q2), in2 = (h2 > p && h2 < q2);
          if (in1 && (!in2 || fabsf(h1) <= fabsf(h2))) h = h1;
          else if (in2) h = h2;
          else ok = false;
        }
      }
    }
    float tn = tau + h;
    if (!ok || !(tn > lo && tn < hi) || !isfinite(tn)) tn = 0.5f * (lo + hi);
    const bool small = fabsf(tn - tau) <= 2e-7f * fabsf(tau);
    tau = tn;
    if (small || (hi - lo) <= 4e-7f * fmaxf(fabsf(lo), fabsf(hi))) break;
  }
  if (o == j ? !(tau > 0.0f && tau < width) : !(tau > -width && tau < 0.0f)) return false;
  org_out = o;
  tau_out = tau;
  return true;
}

// The certified FP64 iteration of secular_certified for one thread: one full pass
// at tau1 keeps the six poles j-2 .. j+3 apart from the far sums (t, t r, t r^2 per
// side), the following iterates re-evaluate only those six; same remainder bound
// and acceptance test.
__device__ bool secular_certified_thread(const double* D, const double* zz, int K, int j, double irho, int org,
                                         double& tau, double& lo, double& hi, bool& conv) {
  const double dorg = D[org];
  const double dl = D[j] - dorg, dr = (j < K - 1) ? D[j + 1] - dorg : 0.0;
  const int wlo = max(0, j - 2), whi = min(K - 1, j + 3);
  const double tau1 = tau;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, b0 = 0.0, b1 = 0.0, b2 = 0.0;
  for (int i = 0; i < wlo; ++i) {
    const double r = rcp_nr((D[i] - dorg) - tau1);
    const double t = zz[i] * r, tr = t * r;
    a0 += t; a1 += tr; a2 = fma(tr, r, a2);
  }
  for (int i = whi + 1; i < K; ++i) {
    const double r = rcp_nr((D[i] - dorg) - tau1);
    const double t = zz[i] * r, tr = t * r;
    b0 += t; b1 += tr; b2 = fma(tr, r, b2);
  }
  double dmin = HUGE_VAL;
  if (wlo - 1 >= 0) dmin = fmin(dmin, fabs((D[wlo - 1] - dorg) - tau1));
  if (whi + 1 < K) dmin = fmin(dmin, fabs((D[whi + 1] - dorg) - tau1));
  // rounding bound of the two recursive far sums (terms of one sign each: at most
  // one unit roundoff of the sum per addition), added to the acceptance threshold
  // so that a root whose |g| is below what this pass can resolve is not rejected
  const double sum_err = kEps * ((double)wlo * fabs(a0) + (double)(K - 1 - whi) * fabs(b0));
  conv = false;
  double tc = tau1;
  for (int k = 0; k < 8; ++k) {
    const double e = tc - tau1;
    const double q = fabs(e) / dmin;
    if (!(q < 4e-6)) break;
    double wl = 0.0, wr = 0.0, wdl = 0.0, wdr = 0.0;
    for (int i = wlo; i <= whi; ++i) {
      const double r = rcp_nr((D[i] - dorg) - tc);
      const double t = zz[i] * r;
      if (i <= j) { wl += t; wdl = fma(t, r, wdl); }
      else { wr += t; wdr = fma(t, r, wdr); }
    }
    const double rest = k > 0 ? (b0 - a0) * (q * q * q) / (1.0 - q) : 0.0;
    const double psi = a0 + e * (a1 + e * a2) + wl, dpsi = a1 + 2.0 * e * a2 + wdl;
    const double phi = b0 + e * (b1 + e * b2) + wr, dphi = b1 + 2.0 * e * b2 + wdr;
    const double gv = irho + psi + phi;
    if (gv == 0.0 || fabs(gv) + rest <= 8.0 * kEps * (irho + (phi - psi)) + sum_err) {
      tau = tc;
      conv = true;
      return true;
    }
    if (fabs(gv) > rest + sum_err) {
      if (gv < 0.0) lo = tc; else hi = tc;
    }
    const double tn = model_step(j, K, irho, dl, dr, tc, gv, psi, dpsi, phi, dphi, lo, hi);
    const bool exact_g = rest <= kEps * (irho + (phi - psi));
    if (exact_g && (fabs(tn - tc) <= 2.0 * kEps * fabs(tc) || (hi - lo) <= 2.0 * kEps * fmax(fabs(lo), fabs(hi)))) {
      tau = tn;
      conv = true;
      return true;
    }
    tc = tn;
  }
  tau = tc;
  return false;
}

// Root j of a small merge by one thread (all poles in its loop): the FP32
// estimate picks the origin and starts the FP64 iteration (whole interval as
// bracket; re-solved from the other pole if it converges in that pole's half);
// without a usable estimate, the origin comes from the sign of g at the midpoint
// and the last root starts from the root of g with the other poles frozen.
// single: only the FP32 estimate and the certified pass; a root that needs more
// (no usable estimate, no certificate, or a root in the other pole's half) comes
// back with conv == false for the warp-per-root solver.
__device__ void secular_root_thread(const double* D, const double* z, const double* zz, const float2* xz,
                                    const float* xlo, int K,
                                    int j, double rho, int max_iter, bool single, int& org_out, double& tau_out,
                                    int& iters, bool& conv) {
  const double irho = 1.0 / rho;
  const bool last = j == K - 1;
  int org;
  double lo, hi, tau, psi, dpsi, phi, dphi, sabs, width;
  if (!last) {
    width = D[j + 1] - D[j];
  } else {
    double zz = 0.0;
    for (int i = 0; i < K; ++i) zz = fma(z[i], z[i], zz);
    width = rho * zz;
  }
  float t32 = 0.0f;
  int o32 = j;
  int passes = 1;
  conv = false;
  org_out = j;
  tau_out = 0.0;
  iters = 1;
  const bool est =
      xz != nullptr && width > 0.0 && secular_fp32_thread(xz, xlo, K, j, (float)irho, (float)width, o32, t32);
  if (single) {
    if (!est) return;
    org = o32;
    tau = (double)t32;
    if (org == j) { lo = 0.0; hi = width; } else { lo = -width; hi = 0.0; }
    if (!(tau > lo && tau < hi)) tau = 0.5 * (lo + hi);
    if (!secular_certified_thread(D, zz, K, j, irho, org, tau, lo, hi, conv)) return;
    if (!last && ((org == j) ? (tau > 0.5 * width) : (tau < -0.5 * width))) {
      conv = false;
      return;
    }
    org_out = org;
    tau_out = tau;
    return;
  }
  if (est) {
    org = o32;
    tau = (double)t32;
    if (org == j) { lo = 0.0; hi = width; } else { lo = -width; hi = 0.0; }
    if (!(tau > lo && tau < hi)) tau = 0.5 * (lo + hi);
    const bool tried = max_iter >= 2;
    if (!tried || !secular_certified_thread(D, zz, K, j, irho, org, tau, lo, hi, conv)) {
      secular_sums<1>(D, z, K, j, D[org], tau, psi, dpsi, phi, dphi, sabs);
      if (tried) ++passes;
      passes += secular_fp64<1>(D, z, K, j, irho, org, tau, lo, hi, psi, dpsi, phi, dphi, sabs, max_iter, conv);
    }
    const bool far = !last && conv && ((org == j) ? (tau > 0.5 * width) : (tau < -0.5 * width));
    if (far) {
      if (org == j) { org = j + 1; tau -= width; lo -= width; hi -= width; }
      else { org = j; tau += width; lo += width; hi += width; }
      secular_sums<1>(D, z, K, j, D[org], tau, psi, dpsi, phi, dphi, sabs);
      ++passes;
      passes += secular_fp64<1>(D, z, K, j, irho, org, tau, lo, hi, psi, dpsi, phi, dphi, sabs, max_iter, conv);
    }
  } else if (!last) {
    secular_sums<1>(D, z, K, j, D[j], 0.5 * width, psi, dpsi, phi, dphi, sabs);
    if (irho + psi + phi >= 0.0) { org = j; lo = 0.0; hi = 0.5 * width; tau = hi; }
    else { org = j + 1; lo = -0.5 * width; hi = 0.0; tau = lo; }
    passes += secular_fp64<1>(D, z, K, j, irho, org, tau, lo, hi, psi, dpsi, phi, dphi, sabs, max_iter, conv);
  } else {
    double s0 = 0.0;
    for (int i = 0; i < j; ++i) s0 += z[i] * z[i] * rcp_nr(D[i] - D[j]);
    org = K - 1; lo = 0.0; hi = width; tau = hi;
    const double den = irho + s0;
    if (den > 0.0) {
      const double t0 = z[j] * z[j] / den;
      if (t0 > lo && t0 < hi) tau = t0;
    }
    secular_sums<1>(D, z, K, j, D[org], tau, psi, dpsi, phi, dphi, sabs);
    passes += secular_fp64<1>(D, z, K, j, irho, org, tau, lo, hi, psi, dpsi, phi, dphi, sabs, max_iter, conv);
  }
  org_out = org;
  tau_out = tau;
  iters = min(passes, max_iter);
}

// Levels with at least kSmallMinSlots slots (many merges, e.g. batches) take
// merges with K <= kSmallK a thread per root: that fills the machine with
// independent work.  Levels with fewer slots keep a warp per root, which finishes
// each root sooner.  small_k is the threshold a launch uses (0: none).
static constexpr int kSmallK = 128;


// Roots of the merges with 0 < K <= small_k, numbered merge by merge: roff[g] is
// the first number of merge g, roff[M] the total (one block, two-level scan).
// Two prefixes over the merges of a level: roff counts the roots of the merges
// with K <= small_k (a thread each), boff the 8-root blocks of the others (a warp
// per root), so that neither kind of kernel visits the other kind's merges.
__global__ void __launch_bounds__(1024) k_root_scan(Plan P, int64_t M, int small_k) {
  __shared__ int64_t part[2][1024];
  const int64_t per = (M + blockDim.x - 1) / blockDim.x;
  const int64_t a = min(M, (int64_t)threadIdx.x * per), b = min(M, a + per);
  int64_t s = 0, sb = 0;
  for (int64_t g = a; g < b; ++g) {
    const int K = P.m.K[g];
    s += (K > 0 && K <= small_k) ? K : 0;
    sb += K > small_k ? (K + 7) / 8 : 0;
  }
  part[0][threadIdx.x] = s;
  part[1][threadIdx.x] = sb;
  __syncthreads();
  if (threadIdx.x < 2) {
    int64_t run = 0;
    for (int i = 0; i < (int)blockDim.x; ++i) {
      const int64_t t = part[threadIdx.x][i];
      part[threadIdx.x][i] = run;
      run += t;
    }
    if (threadIdx.x == 0) {
      P.m.roff[M] = run;
      P.m.roff[M + 1] = 0;  // roots passed on to k_secular_fixup
    } else {
      P.m.boff[M] = run;
    }
  }
  __syncthreads();
  int64_t run = part[0][threadIdx.x], runb = part[1][threadIdx.x];
  for (int64_t g = a; g < b; ++g) {
    P.m.roff[g] = run;
    P.m.boff[g] = runb;
    const int K = P.m.K[g];
    run += (K > 0 && K <= small_k) ? K : 0;
    runb += K > small_k ? (K + 7) / 8 : 0;
  }
}

// The warp-per-root work of a level, as f(g, K, j) for every root j of the merges
// with K > small_k, a warp each.  Merge-major (listed == false): block (g, y) holds
// the roots 8y .. 8y+7 of merge g, and blocks past K or of small merges leave at
// once.  Listed: a fixed grid walks the compacted block list of k_root_scan (on
// levels with many merges, most of the merge-major blocks would be empty).
// A block of fewer than 8 warps takes the 8 roots of its unit in turns.
template <typename F>
__device__ __forceinline__ void for_warp_roots(const Plan& P, int64_t M, int small_k, bool listed, F&& f) {
  const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (!listed) {
    const int64_t g = blockIdx.x;
    const int K = P.m.K[g];
    if (K <= small_k) return;
    for (int u = wid; u < 8; u += nw) {
      const int j = blockIdx.y * 8 + u;
      if (j < K) f(g, K, j);
    }
    return;
  }
  const int64_t total = P.m.boff[M];
  for (int64_t w = blockIdx.x; w < total; w += gridDim.x) {
    int64_t lo = 0, hi = M - 1;
    while (lo < hi) {
      const int64_t m = (lo + hi + 1) >> 1;
      if (P.m.boff[m] <= w) lo = m; else hi = m - 1;
    }
    const int K = P.m.K[lo];
    for (int u = wid; u < 8; u += nw) {
      const int j = (int)(w - P.m.boff[lo]) * 8 + u;
      if (j < K) f(lo, K, j);
    }
  }
}

// Block sizes of the root-side kernels are chosen so that a block fits on an SM
// beside a resident split-GEMM CTA (about 17.9K registers and 59 KB of shared
// memory left): the roots of the next level run while this level's products do.
constexpr int kSecThreads = 128;

static dim3 warp_root_grid(const LevelLaunch& L, bool listed) {
  return listed ? dim3(152 * 8) : dim3((unsigned)L.merges, (unsigned)((L.max_n + 7) / 8));
}

// Thread t -> (merge g, root j) of the small merges: the last g with roff[g] <= t.
__device__ __forceinline__ bool small_root(const Plan& P, int64_t M, int64_t t, int64_t& g, int& j) {
  if (t >= P.m.roff[M]) return false;
  int64_t lo = 0, hi = M - 1;
  while (lo < hi) {
    const int64_t m = (lo + hi + 1) >> 1;
    if (P.m.roff[m] <= t) lo = m; else hi = m - 1;
  }
  g = lo;
  j = (int)(t - P.m.roff[lo]);
  return true;
}

// A thread per root, the FP32 estimate and one certified FP64 pass: a warp waits
// for its slowest lane, so every root that needs more is listed (slot numbers, in
// the sort tag scratch, free between deflation and the final ordering) and
// finished by a warp each in k_secular_fixup.  With an iteration limit below two
// passes the thread runs the whole iteration itself.

__global__ void __launch_bounds__(kSecThreads) k_secular_small(Plan P, int level, int64_t M) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t g;
  int j;
  if (!small_root(P, M, t, g, j)) return;
  const Node nd = make_node(P, level, g);
  const int64_t v0 = nd.v0;
  const int K = P.m.K[g];
  const bool single = P.max_iter >= 2;
  int org, it;
  double tau;
  bool conv;
  secular_root_thread(P.v.Dk + v0, P.v.zk + v0, P.v.zz + v0, P.v.xz + v0, P.v.xlo + v0, K, j, 2.0 * fabs(nd.b),
                      P.max_iter, single, org,
                      tau, it, conv);
  if (!conv && single) {
    const unsigned long long q = atomicAdd(reinterpret_cast<unsigned long long*>(P.m.roff + M + 1), 1ull);
    P.v.stag[q] = (int)(v0 + j);
    return;
  }
  P.v.org[v0 + j] = org;
  P.v.tau[v0 + j] = tau;
  if (!conv) set_status(P.status, TDC_ENOCONV);
  if (P.stats) {
    atomicAdd(&P.stats->iter_sum, (unsigned long long)it);
    atomicAdd(&P.stats->iter_roots, 1ull);
    atomicMax(&P.stats->iter_max, it);
  }
}

// The listed roots, a warp each (the warp-per-root solver with its full budget).
__global__ void __launch_bounds__(kSecThreads) k_secular_fixup(Plan P, int level, int nprob_act, int64_t M) {
  const int64_t cnt = P.m.roff[M + 1];
  if (P.stats && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&P.stats->handoffs, (unsigned long long)cnt);
  for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; w < cnt;
       w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const Slot S = slot_of(P, level, nprob_act, P.v.stag[w]);
    if (!S.valid) continue;
    int org, it;
    double tau;
    bool conv;
    secular_root(P.v.Dk + S.v0, P.v.zk + S.v0, P.v.zz + S.v0, P.v.xz + S.v0, P.v.xlo + S.v0, S.K, S.j, S.rho,
                 P.max_iter, org,
                 tau, it, conv);
    if ((threadIdx.x & 31) == 0) {
      P.v.org[S.v0 + S.j] = org;
      P.v.tau[S.v0 + S.j] = tau;
      if (!conv) set_status(P.status, TDC_ENOCONV);
      if (P.stats) {
        atomicAdd(&P.stats->iter_sum, (unsigned long long)it);
        atomicAdd(&P.stats->iter_roots, 1ull);
        atomicMax(&P.stats->iter_max, it);
      }
    }
  }
}

// Warp per root over the merges with K > small_k (for_warp_roots).
__global__ void __launch_bounds__(kSecThreads) k_secular(Plan P, int level, int64_t M, int small_k, bool listed) {
  for_warp_roots(P, M, small_k, listed, [&](int64_t g, int K, int jw) {
    const Node nd = make_node(P, level, g);
    const int64_t v0 = nd.v0;
    const double rho = 2.0 * fabs(nd.b);
    int org, it;
    double tau;
    bool conv;
    // the merge's first warp takes its last root, usually the slowest to converge,
    // so that it starts with the first wave of warps instead of ending the kernel
    const int j = jw == 0 ? K - 1 : jw - 1;
    secular_root(P.v.Dk + v0, P.v.zk + v0, P.v.zz + v0, P.v.xz + v0, P.v.xlo + v0, K, j, rho, P.max_iter, org, tau,
                 it, conv);
    if ((threadIdx.x & 31) == 0) {
      P.v.org[v0 + j] = org;
      P.v.tau[v0 + j] = tau;
      if (!conv) set_status(P.status, TDC_ENOCONV);
      if (P.stats) {
        atomicAdd(&P.stats->iter_sum, (unsigned long long)it);
        atomicAdd(&P.stats->iter_roots, 1ull);
        atomicMax(&P.stats->iter_max, it);
      }
    }
  });
}

cudaError_t launch_secular(const Plan& P, const LevelLaunch& L, cudaStream_t s) {
  if (L.nslots == 0) return cudaSuccess;
  const int small_k = L.nslots >= kSmallMinSlots ? kSmallK : 0;
  const bool listed = small_k > 0;
  if (listed) k_root_scan<<<1, 512, 0, s>>>(P, L.merges, small_k);
  k_secular<<<warp_root_grid(L, listed), kSecThreads, 0, s>>>(P, L.level, L.merges, small_k, listed);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || small_k == 0) return e;
  k_secular_small<<<(unsigned)((L.nslots + kSecThreads - 1) / kSecThreads), kSecThreads, 0, s>>>(P, L.level,
                                                                                                  L.merges);
  k_secular_fixup<<<152 * 16, kSecThreads, 0, s>>>(P, L.level, L.nprob_act, L.merges);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// k_lowner: zhat_i^2 = prod_j (lambda_j - d_i) / (rho prod_{j != i} (d_j - d_i)),
// with the factors paired as (lambda_j - d_i)/(d_j - d_i) for j < i,
// (lambda_j - d_i)/(d_{j+1} - d_i) for i <= j < K-1 and (lambda_{K-1} - d_i)/rho
// (each ratio in (0, 1]); lambda_j - d_i = (d_org(j) - d_i) + tau_j.
// ---------------------------------------------------------------------------
// Exponent field of x, and x scaled by 2^(1023 - e) (into [1, 2) when e is the
// exponent field of a normal x): integer work plus one multiplication.
__device__ __forceinline__ int dexp_field(double x) { return (__double2hiint(x) >> 20) & 0x7ff; }
__device__ __forceinline__ double dscale(double x, int e) { return x * __hiloint2double((2046 - e) << 20, 0); }

// (x, ex) -> mantissa in [1, 2) and exponent, for normal x (zero, subnormal and
// non-finite values are left as they are)
__device__ __forceinline__ void dnorm(double& x, int& ex) {
  const int f = dexp_field(x);
  if (f > 0 && f < 2047) {
    x = dscale(x, f);
    ex += f - 1023;
  }
}

// The numerator prod_j (lambda_j - d_i) and the denominator prod of the paired
// pole differences are accumulated as two separate products with their exponents
// kept apart (one division per pole instead of one per term): both stay within
// [2^-600, 2^600] and are renormalised when they leave it.
template <int W = 32>
__device__ double lowner_zhat(const double* D, const int* org, const double* tau, int K, int i, double rho,
                              double zsign) {
  const double di = D[i];
  double pn = 1.0, pd = 1.0;
  int en = 0, ed = 0;  // pn 2^en, pd 2^ed
  for (int j = W == 32 ? (threadIdx.x & 31) : 0; j < K; j += W) {
    const double num = (D[org[j]] - di) + tau[j];
    const double den = (j == K - 1) ? rho : ((j < i) ? D[j] - di : D[j + 1] - di);
    pn *= num;
    pd *= den;
    const int fn = dexp_field(pn), fd = dexp_field(pd);
    if (fn < 423 || fn > 1623 || fd < 423 || fd > 1623) {
      dnorm(pn, en);
      dnorm(pd, ed);
    }
  }
  dnorm(pn, en);
  dnorm(pd, ed);
#pragma unroll
  for (int o = 16; o > 0 && W == 32; o >>= 1) {
    const double qn = __shfl_xor_sync(0xffffffffu, pn, o), qd = __shfl_xor_sync(0xffffffffu, pd, o);
    const int gn = __shfl_xor_sync(0xffffffffu, en, o), gd = __shfl_xor_sync(0xffffffffu, ed, o);
    pn *= qn;
    pd *= qd;
    en += gn;
    ed += gd;
    dnorm(pn, en);
    dnorm(pd, ed);
  }
  // zhat_i^2 = (pn / pd) 2^(en - ed), with an even exponent for the root
  double r = pn / pd;
  int E = en - ed;
  if (E & 1) {
    r *= 2.0;
    E -= 1;
  }
  return copysign(ldexp(sqrt(r), E / 2), zsign);
}

__global__ void __launch_bounds__(256) k_lowner(Plan P, int level, int64_t M, int small_k, bool listed) {
  for_warp_roots(P, M, small_k, listed, [&](int64_t g, int K, int j) {
    const Node nd = make_node(P, level, g);
    const int64_t v0 = nd.v0;
    const double zh =
        lowner_zhat(P.v.Dk + v0, P.v.org + v0, P.v.tau + v0, K, j, 2.0 * fabs(nd.b), P.v.zk[v0 + j]);
    if ((threadIdx.x & 31) == 0) P.v.zhat[v0 + j] = zh;
  });
}

// Merges with K <= kSmallK: a thread per pole (k_colnorm_small: per column).
__global__ void __launch_bounds__(256) k_lowner_small(Plan P, int level, int64_t M) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t g;
  int j;
  if (!small_root(P, M, t, g, j)) return;
  const Node nd = make_node(P, level, g);
  const int64_t v0 = nd.v0;
  P.v.zhat[v0 + j] = lowner_zhat<1>(P.v.Dk + v0, P.v.org + v0, P.v.tau + v0, P.m.K[g], j, 2.0 * fabs(nd.b),
                                    P.v.zk[v0 + j]);
}


// s_j = 1 / sqrt(sum_i (zhat_i / delta_ij)^2), delta_ij = (d_i - d_org(j)) - tau_j.
template <int W = 32>
__device__ double column_norm(const double* D, const double* zh, int K, double dorg, double tj) {
  double acc = 0.0;
  for (int i = W == 32 ? (threadIdx.x & 31) : 0; i < K; i += W) {
    const double u = zh[i] * rcp_nr((D[i] - dorg) - tj);
    acc = fma(u, u, acc);
  }
  if (W == 32) acc = warp_sum(acc);
  return 1.0 / sqrt(acc);
}

// The same pass for a merge below the top level, which also forms its boundary
// rows at root j's column: with u_i = zhat_i / delta_ij, Qhat_ij = s_j u_i, so the
// first row there is s_j sum_i pf_i u_i and the last s_j sum_i pl_i u_i (pf, pl:
// the rotated children rows at the poles' columns, zero outside their support) --
// two more multiply-adds per term.  The leftmost node of a level skips the first
// row and the rightmost the last (no merge reads them).
template <int W = 32>
__device__ double column_norm_rows(const Plan& P, int64_t v0, int K, int j, bool need_f, bool need_l) {
  const double* D = P.v.Dk + v0;
  const double* zh = P.v.zhat + v0;
  const double* pf = P.v.pf + v0;
  const double* pl = P.v.pl + v0;
  const double dorg = D[P.v.org[v0 + j]], tj = P.v.tau[v0 + j];
  double acc = 0.0, f = 0.0, l = 0.0;
  const int i0 = W == 32 ? (threadIdx.x & 31) : 0;
  if (need_f && need_l) {
    for (int i = i0; i < K; i += W) {
      const double u = zh[i] * rcp_nr((D[i] - dorg) - tj);
      acc = fma(u, u, acc);
      f = fma(pf[i], u, f);
      l = fma(pl[i], u, l);
    }
  } else {
    const double* pq = need_f ? pf : pl;
    double x = 0.0;
    for (int i = i0; i < K; i += W) {
      const double u = zh[i] * rcp_nr((D[i] - dorg) - tj);
      acc = fma(u, u, acc);
      x = fma(pq[i], u, x);
    }
    if (need_f) f = x; else l = x;
  }
  if (W == 32) {
    acc = warp_sum(acc);
    f = warp_sum(f);
    l = warp_sum(l);
  }
  const double sj = 1.0 / sqrt(acc);
  if (W == 1 || (threadIdx.x & 31) == 0) {
    P.v.rf[v0 + j] = sj * f;
    P.v.rl[v0 + j] = sj * l;
  }
  return sj;
}

__global__ void __launch_bounds__(256) k_colnorm_small(Plan P, int level, int64_t M) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t g;
  int j;
  if (!small_root(P, M, t, g, j)) return;
  const int64_t v0 = make_node(P, level, g).v0;
  const int K = P.m.K[g];
  if (level > 0) {
    const int64_t idx = g & ((((int64_t)1) << level) - 1);
    P.v.scol[v0 + j] = column_norm_rows<1>(P, v0, K, j, idx != 0, idx != (((int64_t)1) << level) - 1);
    return;
  }
  const double* D = P.v.Dk + v0;
  P.v.scol[v0 + j] = column_norm<1>(D, P.v.zhat + v0, K, D[P.v.org[v0 + j]], P.v.tau[v0 + j]);
}

__global__ void __launch_bounds__(256) k_colnorm(Plan P, int level, int64_t M, int small_k, bool listed) {
  for_warp_roots(P, M, small_k, listed, [&](int64_t g, int K, int j) {
    const int64_t v0 = make_node(P, level, g).v0;
    double sj;
    if (level > 0) {
      const int64_t idx = g & ((((int64_t)1) << level) - 1);
      sj = column_norm_rows(P, v0, K, j, idx != 0, idx != (((int64_t)1) << level) - 1);
    } else {
      const double* D = P.v.Dk + v0;
      sj = column_norm(D, P.v.zhat + v0, K, D[P.v.org[v0 + j]], P.v.tau[v0 + j]);
    }
    if ((threadIdx.x & 31) == 0) P.v.scol[v0 + j] = sj;
  });
}

// Stand-alone rank-one eigenproblem (tdc_rank_one, and each term of the band merge): the
// three warp-per-entry stages, after the FP32 copies of the poles for the pre-iteration
// (coordinates relative to the middle pole as sums of two floats, squared weights), as a
// merge level prepares them.
__global__ void __launch_bounds__(256) k_r1_prep(const double* D, const double* z, int K, double* zz, float2* xz,
                                                  float* xlo) {
  const double dc = D[K >> 1];
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < K; j += (int64_t)gridDim.x * blockDim.x) {
    const double zj = z[j];
    const double x = D[j] - dc;
    const float xh = (float)x;
    xz[j] = make_float2(xh, (float)(zj * zj));
    zz[j] = zj * zj;
    xlo[j] = (float)(x - (double)xh);
  }
}

__global__ void __launch_bounds__(256) k_r1_secular(const double* D, const double* z, const double* zz,
                                                     const float2* xz, const float* xlo, int K, double rho,
                                                     int max_iter, int* org, double* tau, int* status) {
  const int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (j >= K) return;
  int o, it;
  double t;
  bool conv;
  secular_root(D, z, zz, xz, xlo, K, (int)j, rho, max_iter, o, t, it, conv);
  if ((threadIdx.x & 31) == 0) {
    org[j] = o;
    tau[j] = t;
    if (!conv) set_status(status, TDC_ENOCONV);
  }
}

__global__ void __launch_bounds__(256) k_r1_lowner(const double* D, const double* z, const int* org,
                                                    const double* tau, int K, double rho, double* zhat) {
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (i >= K) return;
  const double zh = lowner_zhat(D, org, tau, K, (int)i, rho, z[i]);
  if ((threadIdx.x & 31) == 0) zhat[i] = zh;
}

__global__ void __launch_bounds__(256) k_r1_colnorm(const double* D, const int* org, const double* tau,
                                                     const double* zhat, int K, double* s) {
  const int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (j >= K) return;
  const double sj = column_norm(D, zhat, K, D[org[j]], tau[j]);
  if ((threadIdx.x & 31) == 0) s[j] = sj;
}

size_t rank_one_scratch_bytes(int64_t K) {
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t k = (size_t)std::max<int64_t>(K, 1);
  return al(sizeof(double) * k) + al(sizeof(float2) * k) + al(sizeof(float) * k);
}

cudaError_t launch_rank_one(const double* D, const double* z, int64_t K, double rho, int max_iter, int* org,
                            double* tau, double* zhat, double* s, double* zz, float2* xz, float* xlo, int* status,
                            cudaStream_t st) {
  if (K == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((K * 32 + 255) / 256);
  const bool pre = zz && xz && xlo;
  if (pre) k_r1_prep<<<(unsigned)std::min<int64_t>((K + 255) / 256, 4096), 256, 0, st>>>(D, z, (int)K, zz, xz, xlo);
  k_r1_secular<<<blocks, 256, 0, st>>>(D, z, pre ? zz : nullptr, pre ? xz : nullptr, pre ? xlo : nullptr, (int)K,
                                       rho, max_iter, org, tau, status);
  k_r1_lowner<<<blocks, 256, 0, st>>>(D, z, org, tau, (int)K, rho, zhat);
  k_r1_colnorm<<<blocks, 256, 0, st>>>(D, org, tau, zhat, (int)K, s);
  return cudaGetLastError();
}

cudaError_t launch_lowner(const Plan& P, const LevelLaunch& L, cudaStream_t s) {
  if (L.nslots == 0) return cudaSuccess;
  const unsigned tblocks = (unsigned)((L.nslots + 255) / 256);
  const int small_k = L.nslots >= kSmallMinSlots ? kSmallK : 0;
  const bool listed = small_k > 0;  // block list left by launch_secular's k_root_scan
  const dim3 wgrid = warp_root_grid(L, listed);
  k_lowner<<<wgrid, 256, 0, s>>>(P, L.level, L.merges, small_k, listed);
  if (small_k) k_lowner_small<<<tblocks, 256, 0, s>>>(P, L.level, L.merges);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_colnorm<<<wgrid, 256, 0, s>>>(P, L.level, L.merges, small_k, listed);
  if (small_k) k_colnorm_small<<<tblocks, 256, 0, s>>>(P, L.level, L.merges);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Boundary rows.  Each node's first and last eigenvector rows are kept apart
// (P.v.bf, P.v.bl, by output column): the parent's z is made of them, so the
// parent's roots do not need this node's full product.  At a merge, rbf = (first
// row of Q1, 0) and rbl = (0, last row of Q2) take the deflating rotations as
// k_rotate applies them to the columns of diag(Q1, Q2) (row 0 lies in the top
// half, row n-1 in the bottom one); once the roots, zhat, the normalisers and the
// output order are known, the node's rows are these vectors times Qhat for the
// non-deflated columns (the same pole lists and entries as the products) and
// copies for the deflated ones.  The top level has no parent and skips all this.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_boundary_rot(Plan P, int level) {
  const int64_t g = blockIdx.x;
  const Node nd = make_node(P, level, g);
  const int n = (int)(nd.hi - nd.lo), n1 = (int)(nd.mid - nd.lo);
  const int64_t v0 = nd.v0;
  double* rf = P.v.rbf + v0;
  double* rl = P.v.rbl + v0;
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    rf[c] = c < n1 ? P.cbf[v0 + c] : 0.0;
    rl[c] = c < n1 ? 0.0 : P.cbl[v0 + c];
  }
  const int nr = P.m.nrot[g];
  __syncthreads();
  const int nch = nr > 0 ? P.m.nchain[g] : 0;
  for (int h = threadIdx.x; h < nch; h += blockDim.x) {
    const int k0 = P.v.rch[v0 + h];
    const int k1 = (h + 1 < nch) ? P.v.rch[v0 + h + 1] : nr;
    for (int k = k0; k < k1; ++k) {
      const int pj = P.v.rij[4 * (v0 + k) + 0];
      const int ci = P.v.rij[4 * (v0 + k) + 1];
      const int sup = P.v.rij[4 * (v0 + k) + 2];
      const int sp = sup & 0xff, si = sup >> 8;
      const double c = P.v.rcs[2 * (v0 + k)], s = P.v.rcs[2 * (v0 + k) + 1];
      if ((sp | si) & 1) {
        const double x = (sp & 1) ? rf[pj] : 0.0, y = (si & 1) ? rf[ci] : 0.0;
        rf[pj] = c * x + s * y;
        rf[ci] = c * y - s * x;
      }
      if ((sp | si) & 2) {
        const double x = (sp & 2) ? rl[pj] : 0.0, y = (si & 2) ? rl[ci] : 0.0;
        rl[pj] = c * x + s * y;
        rl[ci] = c * y - s * x;
      }
    }
  }
  __syncthreads();
  // by pole: the rotated rows at the pole's column, where the pole has support
  const int K = P.m.K[g];
  for (int i = threadIdx.x; i < K; i += blockDim.x) {
    const int col = P.v.kept[v0 + i];
    const int sup = P.v.kseg[v0 + i];
    P.v.pf[v0 + i] = (sup & 1) ? rf[col] : 0.0;
    P.v.pl[v0 + i] = (sup & 2) ? rl[col] : 0.0;
  }
}

// The node's boundary rows in output order: root j's entries (formed with the
// column norms) go to column posr[j]; deflated entry q copies its (rotated)
// column's entries to column posd[q].
__global__ void __launch_bounds__(256) k_boundary_out(Plan P, int level) {
  const int64_t g = blockIdx.x;
  const int t = blockIdx.y * blockDim.x + threadIdx.x;
  const int K = P.m.K[g];
  const int64_t v0 = make_node(P, level, g).v0;
  if (t < K) {
    const int o = P.v.posr[v0 + t];
    P.v.bf[v0 + o] = P.v.rf[v0 + t];
    P.v.bl[v0 + o] = P.v.rl[v0 + t];
    return;
  }
  const int q = t - K;
  if (q >= P.m.nd[g]) return;
  const int c = P.v.dcol[v0 + q], sp = P.v.dseg[v0 + q], o = P.v.posd[v0 + q];
  P.v.bf[v0 + o] = (sp & 1) ? P.v.rbf[v0 + c] : 0.0;
  P.v.bl[v0 + o] = (sp & 2) ? P.v.rbl[v0 + c] : 0.0;
}

cudaError_t launch_boundary_rot(const Plan& P, const LevelLaunch& L, cudaStream_t s) {
  if (L.level == 0 || L.merges == 0) return cudaSuccess;
  int threads = 256;
  while (threads > 32 && threads / 2 >= L.max_n) threads /= 2;
  k_boundary_rot<<<(unsigned)L.merges, threads, 0, s>>>(P, L.level);
  return cudaGetLastError();
}

cudaError_t launch_boundary_out(const Plan& P, const LevelLaunch& L, cudaStream_t s) {
  if (L.level == 0 || L.nslots == 0) return cudaSuccess;
  k_boundary_out<<<dim3((unsigned)L.merges, (unsigned)((L.max_n + 255) / 256)), 256, 0, s>>>(P, L.level);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// k_finalize: one block per merge.  All n eigenvalues of the node -- the K
// roots d_org(j) + tau_j and the deflated values -- sorted ascending (stable
// over [roots, deflated]) with a bitonic network in the sort scratch; the
// result goes to lam, and every root / deflated entry learns its output column.
// ---------------------------------------------------------------------------
// Doubles as unsigned integers in the same order (negative values with all bits
// flipped, others with the sign bit set), so that the sort compares on the
// integer pipes; NaN is mapped to +infinity first.
__device__ __forceinline__ unsigned long long sort_key(double x) {
  if (isnan(x)) x = INFINITY;
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double key_value(unsigned long long k) {
  return __longlong_as_double((long long)((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k));
}
__device__ __forceinline__ bool key_less(unsigned long long ka, int ta, unsigned long long kb, int tb) {
  return ka < kb || (ka == kb && ta < tb);
}

// Ascending order of the node's eigenvalues: bitonic sort of (value, tag) pairs,
// tags breaking ties (a total order).  Stages whose partners lie within a chunk
// of kSortChunk entries run in shared memory, the wider ones in global memory.
static constexpr int kSortChunk = 2048;

__global__ void __launch_bounds__(1024) k_finalize(Plan P, int level) {
  __shared__ unsigned long long sk[kSortChunk];
  __shared__ int stg[kSortChunk];
  const int64_t g = blockIdx.x;
  const Node nd = make_node(P, level, g);
  const int n = (int)(nd.hi - nd.lo), n1 = (int)(nd.mid - nd.lo);
  const int64_t v0 = nd.v0;
  const int K = P.m.K[g];
  int P2 = 1;
  while (P2 < n) P2 <<= 1;
  unsigned long long* key = reinterpret_cast<unsigned long long*>(P.v.skey + 2 * v0);
  int* tag = P.v.stag + 2 * v0;
  for (int t = threadIdx.x; t < P2; t += blockDim.x) {
    double kv;
    if (t < K) { kv = P.v.Dk[v0 + P.v.org[v0 + t]] + P.v.tau[v0 + t]; tag[t] = t; }
    else if (t < n) { kv = P.v.dval[v0 + t - K]; tag[t] = t; }
    else { kv = INFINITY; tag[t] = 0x7fffffff; }
    key[t] = sort_key(kv);  // the n real entries come first
  }
  __syncthreads();
  const int len = min(P2, kSortChunk);
  // stages k0..k1 (jj from jtop down to 1) of every chunk in shared memory
  auto chunk_stages = [&](int k0, int k1, int jtop) {
    for (int c0 = 0; c0 < P2; c0 += len) {
      for (int t = threadIdx.x; t < len; t += blockDim.x) {
        sk[t] = key[c0 + t];
        stg[t] = tag[c0 + t];
      }
      __syncthreads();
      for (int k = k0; k <= k1; k <<= 1) {
        for (int jj = (k == k0 ? jtop : k >> 1); jj > 0; jj >>= 1) {
          for (int t = threadIdx.x; t < len; t += blockDim.x) {
            const int u = t ^ jj;
            if (u > t) {
              const bool up = ((c0 + t) & k) == 0;
              const unsigned long long ka = sk[t], kb = sk[u];
              const int ta = stg[t], tb = stg[u];
              const bool sw = up ? key_less(kb, tb, ka, ta) : key_less(ka, ta, kb, tb);
              if (sw) { sk[t] = kb; sk[u] = ka; stg[t] = tb; stg[u] = ta; }
            }
          }
          __syncthreads();
        }
      }
      for (int t = threadIdx.x; t < len; t += blockDim.x) {
        key[c0 + t] = sk[t];
        tag[c0 + t] = stg[t];
      }
      __syncthreads();
    }
  };
  if (P2 > 1) chunk_stages(2, len, 1);
  for (int k = 2 * len; k <= P2; k <<= 1) {
    for (int jj = k >> 1; jj >= len; jj >>= 1) {
      for (int t = threadIdx.x; t < P2; t += blockDim.x) {
        const int u = t ^ jj;
        if (u > t) {
          const bool up = (t & k) == 0;
          const unsigned long long ka = key[t], kb = key[u];
          const int ta = tag[t], tb = tag[u];
          const bool sw = up ? key_less(kb, tb, ka, ta) : key_less(ka, ta, kb, tb);
          if (sw) { key[t] = kb; key[u] = ka; tag[t] = tb; tag[u] = ta; }
        }
      }
      __syncthreads();
    }
    chunk_stages(k, k, len >> 1);
  }
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    const int t = tag[p];
    P.v.lam[v0 + p] = key_value(key[p]);
    if (t < K) P.v.posr[v0 + t] = p;
    else if (t < n) P.v.posd[v0 + t - K] = p;
  }
  if (threadIdx.x == 0) {
    // GEMM tiles of this merge: (row tiles of top + bottom parts) x column tiles
    int bm, bn;
    dense_tile_dims(n, bm, bn);
    const int64_t rt = (n1 + bm - 1) / bm + (n - n1 + bm - 1) / bm;
    const int64_t ct = (K + bn - 1) / bn;
    const bool split = P.split_min_K > 0 && K >= P.split_min_K;
    const bool tiny = tiny_merge(n, K, P.m.ntop[g], P.m.nbot[g], P.split_min_K, P.struct_min_K);
    P.m.tiles[g + 1] = (K > 0 && !split && !tiny) ? rt * ct : 0;
  }
}

__global__ void k_tile_scan(Plan P, int64_t M) {
  // single block exclusive scan of P.m.tiles[1..M] into a prefix with tiles[0] = 0
  __shared__ int64_t part[1024];
  const int64_t per = (M + blockDim.x - 1) / blockDim.x;
  const int64_t a = min(M, (int64_t)threadIdx.x * per), b = min(M, a + per);
  int64_t s = 0;
  for (int64_t i = a; i < b; ++i) s += P.m.tiles[i + 1];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t run = 0;
    for (int i = 0; i < (int)blockDim.x; ++i) { int64_t t = part[i]; part[i] = run; run += t; }
  }
  __syncthreads();
  int64_t run = part[threadIdx.x];
  for (int64_t i = a; i < b; ++i) { run += P.m.tiles[i + 1]; P.m.tiles[i + 1] = run; }
  if (threadIdx.x == 0) P.m.tiles[0] = 0;
}

cudaError_t launch_finalize(const Plan& P, const LevelLaunch& L, cudaStream_t s) {
  int threads = 512;
  while (threads > 64 && threads / 2 >= L.max_n) threads /= 2;
  k_finalize<<<(unsigned)L.merges, threads, 0, s>>>(P, L.level);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_tile_scan<<<1, 512, 0, s>>>(P, L.merges);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// k_copy_defl: deflated eigenvectors (columns of the rotated Q) to their output
// columns; entries outside the column's row support are written as zeros.
// ---------------------------------------------------------------------------
// Warp w of block (g, y, z) copies rows [y*kCopyRows, (y+1)*kCopyRows) of the
// deflated columns z*8+w, z*8+w + 8*gridDim.z, ... of merge g: rows and columns
// are both spread over the grid, so a few long columns and many short ones both
// fill the machine.
static constexpr int kCopyRows = 2048;

__global__ void __launch_bounds__(256) k_copy_defl(Plan P, int level) {
  const int64_t g = blockIdx.x;
  const int ndf = P.m.nd[g];
  if (ndf == 0) return;
  const Node nd = make_node(P, level, g);
  const int n = (int)(nd.hi - nd.lo), n1 = (int)(nd.mid - nd.lo);
  const int r0 = blockIdx.y * kCopyRows;
  if (r0 >= n) return;
  const int r1 = min(n, r0 + kCopyRows);
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int64_t v0 = nd.v0;
  for (int q = blockIdx.z * nw + (threadIdx.x >> 5); q < ndf; q += gridDim.z * nw) {
    const int c = P.v.dcol[v0 + q];
    const int sp = P.v.dseg[v0 + q];
    const int o = P.v.posd[v0 + q];
    if (o < 0 || o >= n) continue;
    const double* src = nd.src + (int64_t)c * nd.lds;
    double* dst = nd.dst + (int64_t)o * nd.ldd;
#pragma unroll 8
    for (int r = r0 + lane; r < r1; r += 32) {
      const int half = r < n1 ? 1 : 2;
      dst[r] = (sp & half) ? src[r] : 0.0;
    }
  }
}

// The top merge of each problem (level 0) writes the caller's Q: there a warp owns
// a whole deflated column, finds its entry of largest magnitude within the
// column's row support (lowest row on ties, as the output pass does) and writes
// the column with the sign convention already applied, so that the output pass
// can skip it.  Magnitudes compare as integers of their bits.
__global__ void __launch_bounds__(256) k_copy_defl_sign(Plan P) {
  const int64_t g = blockIdx.x;
  const int ndf = P.m.nd[g];
  if (ndf == 0) return;
  const Node nd = make_node(P, 0, g);
  const int n = (int)(nd.hi - nd.lo), n1 = (int)(nd.mid - nd.lo);
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int64_t v0 = nd.v0;
  for (int q = blockIdx.y * nw + (threadIdx.x >> 5); q < ndf; q += gridDim.y * nw) {
    const int c = P.v.dcol[v0 + q];
    const int sp = P.v.dseg[v0 + q];
    const int o = P.v.posd[v0 + q];
    if (o < 0 || o >= n) continue;
    const int ra = (sp & 1) ? 0 : n1, rb = (sp & 2) ? n : n1;  // row support [ra, rb)
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(nd.src + (int64_t)c * nd.lds);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(nd.dst + (int64_t)o * nd.ldd);
    unsigned long long best = 0ull;
    int bi = ra;
    bool any = false;
    for (int r0 = ra; r0 < rb; r0 += 256) {
      unsigned long long v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int r = r0 + k * 32 + lane;
        v[k] = r < rb ? (src[r] & 0x7fffffffffffffffull) : 0ull;
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int r = r0 + k * 32 + lane;
        if (r < rb && v[k] <= 0x7ff0000000000000ull && (!any || v[k] > best)) { best = v[k]; bi = r; any = true; }
      }
    }
    for (int off = 16; off > 0; off >>= 1) {
      const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, off);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
      const bool oa = __shfl_xor_sync(0xffffffffu, any, off);
      if (oa && (!any || ob > best || (ob == best && oi < bi))) { best = ob; bi = oi; any = true; }
    }
    const unsigned long long flip = (rb > ra && (long long)src[bi] < 0) ? 0x8000000000000000ull : 0ull;
    for (int r0 = 0; r0 < n; r0 += 256) {
      unsigned long long v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int r = r0 + k * 32 + lane;
        v[k] = (r >= ra && r < rb) ? src[r] ^ flip : 0ull;
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int r = r0 + k * 32 + lane;
        if (r < n) dst[r] = v[k];
      }
    }
  }
}

cudaError_t launch_copy_deflated(const Plan& P, const LevelLaunch& L, int sign_normalise, cudaStream_t s) {
  if (L.level == 0 && sign_normalise) {
    const unsigned gy = (unsigned)std::max<int64_t>(1, std::min<int64_t>(1024, L.max_n / 64));
    k_copy_defl_sign<<<dim3((unsigned)L.merges, gy), 256, 0, s>>>(P);
    return cudaGetLastError();
  }
  const unsigned gy = (unsigned)((L.max_n + kCopyRows - 1) / kCopyRows);
  const unsigned gz = (unsigned)std::max<int64_t>(1, std::min<int64_t>(256, L.max_n / 64));
  dim3 grid((unsigned)L.merges, gy, gz);
  k_copy_defl<<<grid, 256, 0, s>>>(P, L.level);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Output: sign convention (entry of largest magnitude positive, lowest row on
// ties) and eigenvalues to the caller's array.  One warp per column.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_sign_out(Plan P, int sign_normalise) {
  const int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (s >= P.nslots) return;
  const int lane = threadIdx.x & 31;
  const int pi = find_problem_by_slot(P.prob, P.nprob, s);
  const Problem& p = P.prob[pi];
  const int64_t c = s - p.voff;
  double* col = P.Q0 + p.off_q + c * p.ld0;
  // columns of the top merge that came from deflation were normalised by the copy
  const bool done = p.depth > 0 && P.v.stag[2 * p.voff + c] >= P.m.K[pi];
  if (sign_normalise && !done) {
    // |x| compared as the integer of its bits (same order for finite values, on the
    // integer pipes); eight independent loads per lane in flight
    const unsigned long long* cb = reinterpret_cast<const unsigned long long*>(col);
    unsigned long long best = 0ull;
    int64_t bi = 0;
    bool any = false;
    for (int64_t r0 = 0; r0 < p.n; r0 += 256) {
      unsigned long long v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int64_t r = r0 + k * 32 + lane;
        v[k] = r < p.n ? (cb[r] & 0x7fffffffffffffffull) : 0ull;
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int64_t r = r0 + k * 32 + lane;
        if (r < p.n && v[k] <= 0x7ff0000000000000ull && (!any || v[k] > best)) { best = v[k]; bi = r; any = true; }
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int64_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
      const bool oa = __shfl_xor_sync(0xffffffffu, any, o);
      if (oa && (!any || ob > best || (ob == best && oi < bi))) { best = ob; bi = oi; any = true; }
    }
    if ((long long)cb[bi] < 0) {  // sign bit of the largest entry
      unsigned long long* cw = reinterpret_cast<unsigned long long*>(col);
      for (int64_t r0 = 0; r0 < p.n; r0 += 256) {
        unsigned long long v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int64_t r = r0 + k * 32 + lane;
          v[k] = r < p.n ? cw[r] : 0ull;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int64_t r = r0 + k * 32 + lane;
          if (r < p.n) cw[r] = v[k] ^ 0x8000000000000000ull;
        }
      }
    }
  }
  if (lane == 0) P.lam_out[p.off_de + c] = p.escale ? scale2(P.v.lam[s], p.escale) : P.v.lam[s];
}

cudaError_t launch_sign_and_output(const Plan& P, int sign_normalise, cudaStream_t s) {
  if (P.nslots == 0) return cudaSuccess;
  const int64_t blocks = (P.nslots * 32 + 255) / 256;
  k_sign_out<<<(unsigned)blocks, 256, 0, s>>>(P, sign_normalise);
  return cudaGetLastError();
}

}  // namespace tdc
