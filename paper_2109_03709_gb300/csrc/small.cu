// small.cu -- the small dense kernels of the pPCA path (d x m and m x m work).
//
//   gram_df          G = A^T B with double-float accumulation (CholeskyQR2's Gram,
//                    the projected Gram of the pPCA step, Oja's Y^T Y, EigenGame's C)
//   cholesky_adaptive G = R^T R and R^-1: blocked FP32 on the diagonally scaled
//                    G, double-float fallback when the conditioning bound fails
//                    -- CholeskyQR2
//   apply_rinv       Q = V R^-1                                   -- CholeskyQR2
//   eigh_small       parallel-order Jacobi (FP32 sweeps) + FP64 Rayleigh quotients
//                    -- the full-PCA of Algorithm 1, step 4
//   rotate_and_sign  E = Q U[:, :k], sign convention, lambda = w / n -- step 5
//   oja_update       generalised Oja (Sanger) rule, Section 2.2
//   eigengame_update EigenGame utility gradients (Section 2.3, Eq. 3), Riemannian
//                    projection, Nesterov momentum (Section 5), renormalisation
//   init_gaussian    Philox4x32-10 + Box-Muller starting basis
//   quantize_*       BF16 / FP8 E4M3 data formats
#include "kernels.h"
#include "grouped.h"

#include <cuda_fp8.h>
#include <math.h>

#include <algorithm>
#include <map>
#include <mutex>

namespace ppca {

namespace {

constexpr int kGramTile = 32;        // output tile of gram_df
constexpr int kGramRows = 32;        // rows of A/B per slice (one tile of 32 rows)

// Row slices of gram_df: one per kGramRows rows, at most 1024 / T^2 (at least
// 128) for T x T output tiles, so that a narrow basis over many rows still
// fills the GPU.
inline int gram_nslices(int64_t d, int m) {
    const int T = (m + kGramTile - 1) / kGramTile;
    const int cap = 1024 / (T * T) > 128 ? 1024 / (T * T) : 128;
    const int64_t p = (d + kGramRows - 1) / kGramRows;
    return p < 1 ? 1 : (p > cap ? cap : (int)p);
}

// Threads that reduce one output of gram_reduce_kernel: a power of two up to
// 32 leaving each at least four partials.
inline int gram_reduce_lanes(int P) {
    int L = 1;
    while (L < 32 && P / (2 * L) >= 4) L *= 2;
    return L;
}

// Exact product of two floats as an unevaluated sum p + e (FMA-based TwoProduct).
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

__device__ __forceinline__ void gram_df_body(const float* __restrict__ A, const float* __restrict__ B, int64_t d,
                                             int m, float* __restrict__ part, int64_t slice_rows, int ti, int tj,
                                             int p) {
    __shared__ float As[32][kGramTile + 1];
    __shared__ float Bs[32][kGramTile + 1];
    if (A == B && ti > tj) return;          // symmetric: the reduction mirrors the upper tiles
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int i0 = ti * kGramTile, j0 = tj * kGramTile;
    const int64_t rbeg = (int64_t)p * slice_rows;
    const int64_t rend = min(d, rbeg + slice_rows);
    float hi[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, lo[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
    for (int64_t r0 = rbeg; r0 < rend; r0 += 32) {
        for (int e = threadIdx.x; e < 32 * kGramTile; e += blockDim.x) {
            const int rr = e % 32, cc = e / 32;
            const int64_t r = r0 + rr;
            const int ia = i0 + cc, jb = j0 + cc;
            As[rr][cc] = (r < rend && ia < m) ? A[(int64_t)ia * d + r] : 0.f;
            Bs[rr][cc] = (r < rend && jb < m) ? B[(int64_t)jb * d + r] : 0.f;
        }
        __syncthreads();
        // Dot2 over the 32 rows of the tile (Ogita, Rump and Oishi, "Accurate
        // sum and dot product", 2005): the running sum sacc carries one
        // rounding per step, whose exact error (TwoSum) and the product's
        // (TwoProduct) go to cacc; the tile's sacc + cacc is as accurate as a
        // dot product in twice the precision, and is folded into (hi, lo).
        float sacc[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, cacc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll 8
        for (int rr = 0; rr < 32; ++rr) {
#pragma unroll
            for (int a = 0; a < 2; ++a) {
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    float pp, pe, sn, se;
                    two_prod(As[rr][ty * 2 + a], Bs[rr][tx * 2 + b], pp, pe);
                    two_sum(sacc[a][b], pp, sn, se);
                    sacc[a][b] = sn;
                    cacc[a][b] = __fadd_rn(cacc[a][b], __fadd_rn(se, pe));
                }
            }
        }
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                df_add(hi[a][b], lo[a][b], sacc[a][b]);
                lo[a][b] = __fadd_rn(lo[a][b], cacc[a][b]);
            }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int i = i0 + ty * 2 + a, j = j0 + tx * 2 + b;
            if (i < m && j < m) {
                float* o = part + (((int64_t)p * m + i) * m + j) * 2;
                o[0] = hi[a][b];
                o[1] = lo[a][b];
            }
        }
}

__global__ void gram_df_kernel(const float* __restrict__ A, const float* __restrict__ B, int64_t d, int m,
                               float* __restrict__ part, int64_t slice_rows, const int* run_if) {
    if (run_if && *run_if == 0) return;       // only needed when the FP32 factorisation was rejected
    gram_df_body(A, B, d, m, part, slice_rows, blockIdx.x, blockIdx.y, blockIdx.z);
}

// L consecutive threads (L a power of two dividing 32) reduce one output: lane
// l sums slices l, l + L, ... in order, then the lanes are combined by a fixed
// shuffle tree, all in double-float.
__device__ __forceinline__ void gram_reduce_body(const float* __restrict__ part, int P, int m, int L, bool sym,
                                                 double* __restrict__ G, float* __restrict__ Gf, int block) {
    const int64_t g = (int64_t)block * blockDim.x + threadIdx.x;
    const int idx = (int)(g / L), lane = (int)(g % L);
    const bool live = idx < m * m;               // whole groups are live or not: shuffles stay uniform
    dfloat q = {0.f, 0.f};
    if (live) {
        const int i = idx / m, j = idx % m;
        const int src = (sym && i / kGramTile > j / kGramTile) ? j * m + i : idx;
        for (int p = lane; p < P; p += L) {
            const float2 o = reinterpret_cast<const float2*>(part)[(int64_t)p * m * m + src];
            q = df_addx(q, df_norm(o.x, o.y));
        }
    }
    for (int o = L / 2; o > 0; o >>= 1) {
        dfloat r;
        r.hi = __shfl_down_sync(0xffffffffu, q.hi, o, L);
        r.lo = __shfl_down_sync(0xffffffffu, q.lo, o, L);
        q = df_addx(q, r);
    }
    if (live && lane == 0) {
        G[idx] = (double)q.hi + (double)q.lo;
        if (Gf) Gf[idx] = q.hi;
    }
}

__global__ void gram_reduce_kernel(const float* __restrict__ part, int P, int m, int L, bool sym,
                                   double* __restrict__ G, float* __restrict__ Gf, const int* run_if) {
    if (run_if && *run_if == 0) return;
    gram_reduce_body(part, P, m, L, sym, G, Gf, blockIdx.x);
}

// ------------------------------------------------------------------ Cholesky

// Right-looking Cholesky G = R^T R (R upper) in one CTA, then the triangular
// inverse X = R^-1 in FP32, written row-major to Rinv.  DF = true works in
// double-float arithmetic -- FP64-class accuracy (about 48 significand bits)
// at FP32-pipe speed, for the first, possibly ill-conditioned CholeskyQR pass;
// DF = false is plain FP32 for the second pass, whose Gram matrix is within
// rounding of the identity.  A pivot at or below 1e-15 * trace(G) (also NaN)
// marks the basis as numerically rank-deficient: the pivot is replaced by that
// floor (so the outputs stay finite) and kDevCholeskyBreakdown is recorded.
// Thread layout: warp w handles rows i = k+1+w, k+1+w+W, ...; lanes sweep
// the columns j >= i of that row (no integer division in the inner loops).
constexpr int kCholThreads = 512;

template <bool DF>
__device__ __forceinline__ void cholesky_body(const double* __restrict__ G, int m, float* __restrict__ Rinv,
                                              int* status) {
    extern __shared__ float csm[];
    float* ah = csm;                       // m x m, hi parts (the FP32 value when !DF)
    float* al = ah + m * m;                // m x m, lo parts (DF only)
    float* x = DF ? al + m * m : al;       // m x m: R (row-major), then overwritten by R^-1
    __shared__ float inv_hi, inv_lo, floor_pivot;
    __shared__ int broke;
    const int lane = threadIdx.x % 32, warp = threadIdx.x / 32, nw = kCholThreads / 32;
    for (int e = threadIdx.x; e < m * m; e += kCholThreads) {
        const dfloat v = df_make(G[e]);
        ah[e] = v.hi;
        if (DF) al[e] = v.lo;
    }
    if (warp == 0) {
        double tr = 0.0;
        for (int i = lane; i < m; i += 32) tr += fabs(G[i * m + i]);
        for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
        if (lane == 0) {
            floor_pivot = (float)((tr > 0.0 ? tr : 1.0) * 1e-15);
            broke = 0;
        }
    }
    __syncthreads();
    for (int k = 0; k < m; ++k) {
        if (threadIdx.x == 0) {
            dfloat pv{ah[k * m + k], DF ? al[k * m + k] : 0.f};
            if (!(pv.hi > floor_pivot)) {   // also catches NaN
                broke = 1;
                pv = dfloat{floor_pivot, 0.f};
            }
            if (DF) {
                const dfloat r = df_sqrtx(pv);
                x[k * m + k] = r.hi;
                const dfloat inv = df_divx(dfloat{1.f, 0.f}, r);
                inv_hi = inv.hi;
                inv_lo = inv.lo;
            } else {
                const float r = sqrtf(pv.hi);
                x[k * m + k] = r;
                inv_hi = 1.0f / r;
                inv_lo = 0.f;
            }
        }
        __syncthreads();
        // row k of R (scaled copy, written to x) and the trailing update
        // a_ij -= r_ki r_kj, k < i <= j, with r_k* = a_k* / r_kk on the fly
        const dfloat inv{inv_hi, inv_lo};
        if (warp == nw - 1)
            for (int j = k + 1 + lane; j < m; j += 32)
                x[k * m + j] = DF ? df_mulx(dfloat{ah[k * m + j], al[k * m + j]}, inv).hi : ah[k * m + j] * inv_hi;
        for (int i = k + 1 + warp; i < m; i += nw) {
            const dfloat rki = DF ? df_mulx(dfloat{ah[k * m + i], al[k * m + i]}, inv)
                                  : dfloat{ah[k * m + i] * inv_hi, 0.f};
            for (int j = i + lane; j < m; j += 32) {
                if (DF) {
                    const dfloat rkj = df_mulx(dfloat{ah[k * m + j], al[k * m + j]}, inv);
                    const dfloat v = df_addx(dfloat{ah[i * m + j], al[i * m + j]}, df_neg(df_mulx(rki, rkj)));
                    ah[i * m + j] = v.hi;
                    al[i * m + j] = v.lo;
                } else {
                    ah[i * m + j] = __fmaf_rn(-rki.hi, ah[k * m + j] * inv_hi, ah[i * m + j]);
                }
            }
        }
        __syncthreads();
    }
    // R (FP32, upper, in x) -> R^-1 in place of ah, row by row from the bottom:
    // row i of X = (e_i - sum_{l>i} r_il X[l, :]) / r_ii; columns in parallel.
    float* X = ah;
    for (int i = m - 1; i >= 0; --i) {
        const float rii = x[i * m + i];
        for (int j = threadIdx.x; j < m; j += kCholThreads) {
            float s = (j == i) ? 1.f : 0.f;
            if (j > i) {
                float s0 = 0.f, s1 = 0.f;
                int l = i + 1;
                for (; l + 1 <= j; l += 2) {
                    s0 = __fmaf_rn(-x[i * m + l], X[l * m + j], s0);
                    s1 = __fmaf_rn(-x[i * m + l + 1], X[(l + 1) * m + j], s1);
                }
                if (l <= j) s0 = __fmaf_rn(-x[i * m + l], X[l * m + j], s0);
                s = s0 + s1;
            }
            X[i * m + j] = (j >= i) ? s / rii : 0.f;
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < m * m; e += kCholThreads) Rinv[e] = X[e];
    if (threadIdx.x == 0 && broke) set_status(status, kDevCholeskyBreakdown);
}

template <bool DF>
__global__ void __launch_bounds__(kCholThreads) cholesky_kernel(const double* __restrict__ G, int m,
                                                               float* __restrict__ Rinv, const int* run_if,
                                                               int* status) {
    if (run_if && *run_if == 0) return;      // the FP32 attempt was accepted
    cholesky_body<DF>(G, m, Rinv, status);
}

// Blocked Cholesky in FP32 of the diagonally scaled Gram matrix G' = D G D
// (D = diag(G)^-1/2, so G' has a unit diagonal), with the triangular inverse
// W = R'^-1; writes Rinv = D W, so V Rinv = V R^-1 for G = R^T R.
//   * near_identity (second CholeskyQR pass): when max|G' - I| <= kSeriesMax
//     the factor comes from the series below (chol_series) and nothing else runs;
//   * otherwise R' by a right-looking blocked Cholesky on 4 x 4 blocks held in
//     registers (two barriers per four columns, described at the loop);
//   * W's 32 x 32 diagonal blocks by back substitution, one warp per block,
//     then its off-diagonal blocks one block diagonal at a time:
//     W_pq = -W_pp sum_{p<l<=q} R_pl W_lq.
// With `fallback` set (first CholeskyQR pass, V possibly ill-conditioned) the
// kernel bounds kappa(G') <= (max row sum |G'|) ||W||_F^2 (Gershgorin for
// lambda_max; trace(G'^-1) = ||W||_F^2 >= 1/lambda_min).  A non-positive
// pivot or a bound above 2^16 sets *fallback = 1 and the double-float kernel
// redoes the factorisation.  2^16 is below 1 / (m u) for every m <= 128: an
// exactly rank-deficient G' rounded to FP32 has lambda_min ~ m u lambda_max,
// so it cannot pass and its breakdown is reported by the double-float kernel;
// an accepted G' has kappa(V D) <= 256, well inside the range where an FP32
// first pass lets the second CholeskyQR pass restore orthogonality.
// Without `fallback` (second pass, G' within rounding of I) a non-positive
// pivot is recorded as kDevCholeskyBreakdown.
constexpr int kCBThreads = 512;
static_assert(kCBThreads == kCholThreads, "the grouped factor kernel runs the fallback in the same block");
constexpr int kCB = 32;
constexpr float kCholKappaMax = 65536.f;     // 2^16
// An accepted first-pass factor whose bound is at most 2^10 leaves Q^T Q within
// about 1e-4 of I: when only span(Q) matters (a block power step) the second
// CholeskyQR pass is skipped (*next = 0).
constexpr float kCholSkipMax = 1024.f;

// C (m x m, upper part, row stride lda) = op(X) Y for upper-triangular X and Y
// on 4 x 4 register tiles: TRANS_X: C = X^T Y (both read by rows); else C = X Y.
// Block-wide; the caller synchronises before and after.
template <bool TRANS_X>
__device__ void upper_matmul(const float* X, const float* Y, float* C, int m, int lda) {
    const int nq = (m + 3) / 4;
    for (int e = threadIdx.x; e < nq * nq; e += blockDim.x) {
        const int bi = e / nq, bj = e % nq;
        if (bi > bj) continue;
        const int i0 = bi * 4, j0 = bj * 4;
        float acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
        const int l0 = TRANS_X ? 0 : i0, l1 = TRANS_X ? min(m, i0 + 4) : min(m, j0 + 4);
        for (int l = l0; l < l1; ++l) {
            float xv[4];
            if (TRANS_X) {
                const float4 x4 = *reinterpret_cast<const float4*>(X + l * lda + i0);
                xv[0] = x4.x; xv[1] = x4.y; xv[2] = x4.z; xv[3] = x4.w;
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) xv[u] = (i0 + u < m) ? X[(i0 + u) * lda + l] : 0.f;
            }
            const float4 y4 = *reinterpret_cast<const float4*>(Y + l * lda + j0);
            const float yv[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = __fmaf_rn(xv[u], yv[v], acc[u][v]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (i0 + u < m)
                *reinterpret_cast<float4*>(C + (i0 + u) * lda + j0) =
                    make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
    }
}

// Second CholeskyQR pass: G' = I + E with small E (the first pass already
// orthonormalised V up to rounding amplified by its conditioning).  Then
// R' = I + N to third order in E, with N = U1 + U2: U1 = the upper triangle of
// E with its diagonal halved, U2 the same of -U1^T U1 (from (I + N)^T (I + N)
// = I + E); and R'^-1 = I - N + N^2 - N^3.  Neglected terms are O(|E|^3) =
// below 1e-8 for |E|_max <= 2e-3, the acceptance bound.  Every step is a
// parallel matrix product instead of m sequential pivots.  Returns false
// (leaving A untouched) when |E|_max is above the bound.
constexpr float kSeriesMax = 2e-3f;

__device__ bool chol_series(float* A, float* W, const float* dsc, int m, int lda, float* __restrict__ Rinv) {
    __shared__ float emax_w[kCBThreads / 32];
    __shared__ int accept;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float mx = 0.f;
    for (int e = tid; e < m * lda; e += blockDim.x) {
        const int i = e / lda, j = e % lda;
        if (j < m) mx = fmaxf(mx, fabsf(A[e] - (i == j ? 1.f : 0.f)));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) emax_w[warp] = mx;
    __syncthreads();
    if (tid == 0) {
        float r = 0.f;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) r = fmaxf(r, emax_w[w]);
        accept = (r <= kSeriesMax) ? 1 : 0;      // false for NaN
    }
    __syncthreads();
    if (!accept) return false;
    // W = U1
    for (int e = tid; e < m * lda; e += blockDim.x) {
        const int i = e / lda, j = e % lda;
        W[e] = (j < m && i < j) ? A[e] : (i == j ? 0.5f * (A[e] - 1.f) : 0.f);
    }
    __syncthreads();
    upper_matmul<true>(W, W, A, m, lda);         // A = U1^T U1 (upper part)
    __syncthreads();
    for (int e = tid; e < m * lda; e += blockDim.x) {   // W = N = U1 + U2
        const int i = e / lda, j = e % lda;
        if (j < m && i < j) W[e] -= A[e];
        else if (i == j) W[e] -= 0.5f * A[e];
    }
    __syncthreads();
    upper_matmul<false>(W, W, A, m, lda);        // A = N^2
    __syncthreads();
    // Rinv = D (I - N + N^2 - N^3), N^3 = N N^2 on the fly
    const int nq = (m + 3) / 4;
    for (int e = tid; e < nq * nq; e += blockDim.x) {
        const int bi = e / nq, bj = e % nq;
        const int i0 = bi * 4, j0 = bj * 4;
        float acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
        if (bi <= bj) {
            for (int l = i0; l < min(m, j0 + 4); ++l) {
                float xv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) xv[u] = (i0 + u < m) ? W[(i0 + u) * lda + l] : 0.f;
                const float4 y4 = *reinterpret_cast<const float4*>(A + l * lda + j0);
                const float yv[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] = __fmaf_rn(xv[u], yv[v], acc[u][v]);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u;
            if (i >= m) continue;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int j = j0 + v;
                if (j >= m) continue;
                float r = 0.f;
                if (i <= j) r = (i == j ? 1.f : 0.f) - W[i * lda + j] + A[i * lda + j] - acc[u][v];
                Rinv[i * m + j] = dsc[i] * r;
            }
        }
    }
    return true;
}

__device__ __forceinline__ void chol_blocked_body(const float* __restrict__ Gf, int m, float* __restrict__ Rinv,
                                                  int* fallback, int* status, int near_identity,
                                                  int* next = nullptr) {
    extern __shared__ __align__(16) float cbs[];
    const int lda = (m + 3) & ~3;           // shared-memory row stride: rows start 16-byte aligned
    float* A = cbs;                         // m x lda; upper triangle, rows of R' overwrite it panel by panel
    float* W = A + m * lda;                 // m x lda, R'^-1 (upper, zero below)
    float* T = W + m * lda;                 // (kCB x kCB) per block pair of one block diagonal (<= nb - 1 pairs)
    float* dsc = T + ((m + kCB - 1) / kCB) * kCB * kCB;   // m: G_ii^-1/2
    __shared__ int bad;
    __shared__ float red[kCBThreads / 32];
    __shared__ float rowsum_max;
    const unsigned full = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nw = kCBThreads / 32;
    const int nb = (m + kCB - 1) / kCB;
    if (tid == 0) bad = 0;
    for (int i = tid; i < m; i += kCBThreads) {
        const float g = Gf[i * m + i];
        dsc[i] = g > 0.f ? __fdiv_rn(1.f, __fsqrt_rn(g)) : 0.f;
    }
    __syncthreads();
    {
        float mx = 0.f;
        for (int i = warp; i < m; i += nw) {
            const float di = dsc[i];
            float sum = 0.f;
            for (int j = lane; j < lda; j += 32) {
                const float v = j < m ? Gf[i * m + j] * di * dsc[j] : 0.f;
                A[i * lda + j] = v;
                W[i * lda + j] = 0.f;
                sum += fabsf(v);
            }
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(full, sum, o);
            mx = fmaxf(mx, sum);
        }
        if (lane == 0) red[warp] = mx;
        __syncthreads();
        if (tid == 0) {
            float r = 0.f;
            for (int w = 0; w < nw; ++w) r = fmaxf(r, red[w]);
            rowsum_max = r;
        }
    }
    if (near_identity && chol_series(A, W, dsc, m, lda, Rinv)) {
        if (tid == 0 && fallback) *fallback = 0;
        return;
    }
    // Right-looking blocked Cholesky G' = R^T R (R upper) with the upper triangle
    // held in registers: the 4 x 4 blocks (bi <= bj) are dealt to the threads, one
    // or two each.  Block step kb: the owner of the diagonal block factors it
    // alone (four pivots, in registers) and writes R_kk and 1 / diag(R_kk) to
    // shared memory; after a barrier the owners of block row kb solve
    // R_kb,j = R_kk^-T A_kb,j for their blocks and write them into A; after a
    // second barrier every thread applies the rank-4 update A_ij -= R_kb,i^T R_kb,j
    // to its blocks below block row kb, and the owner of the next diagonal block
    // factors it right after its own update.  Two barriers per four columns.
    // Rows at or past m (the padding of the last block) are never read or
    // written; their R entries count as zero.
    {
        __shared__ float sh_rinv[4];
        const int nq = (m + 3) / 4;
        const int nblk = nq * (nq + 1) / 2;
        int bI[2], bJ[2];
        float a[2][4][4];
#pragma unroll
        for (int s2 = 0; s2 < 2; ++s2) {
            const int b = tid + s2 * kCBThreads;
            bI[s2] = -1;
            bJ[s2] = 0;
            if (b < nblk) {
                int bi = 0, rem = b;
                while (rem >= nq - bi) {
                    rem -= nq - bi;
                    ++bi;
                }
                bI[s2] = bi;
                bJ[s2] = bi + rem;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int ii = 4 * bI[s2] + u, jj = 4 * bJ[s2] + v;
                    a[s2][u][v] = (bI[s2] >= 0 && ii < m && jj < m) ? A[ii * lda + jj] : 0.f;
                }
        }
        __syncthreads();                      // blocks loaded: A now receives the rows of R
        // factor diagonal block kb in place (the caller owns it, slot s2) and publish it
        auto factor_diag = [&](int s2, int kb) {
            const int k0 = 4 * kb;
            float rd[4][4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
#pragma unroll
                for (int v = 0; v < 4; ++v) rd[c][v] = 0.f;
                float inv = 0.f;
                if (k0 + c < m) {
                    float piv = a[s2][c][c];
                    if (!(piv > 0.f)) {
                        piv = 1e-30f;
                        bad = 1;
                    }
                    const float r = __fsqrt_rn(piv);
                    inv = __frcp_rn(r);
                    rd[c][c] = r;
#pragma unroll
                    for (int v = c + 1; v < 4; ++v) rd[c][v] = a[s2][c][v] * inv;
#pragma unroll
                    for (int u = c + 1; u < 4; ++u)
#pragma unroll
                        for (int v = u; v < 4; ++v) a[s2][u][v] = __fmaf_rn(-rd[c][u], rd[c][v], a[s2][u][v]);
                }
                sh_rinv[c] = inv;
            }
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (k0 + c < m) *reinterpret_cast<float4*>(A + (k0 + c) * lda + k0) =
                                    make_float4(rd[c][0], rd[c][1], rd[c][2], rd[c][3]);
        };
#pragma unroll
        for (int s2 = 0; s2 < 2; ++s2)
            if (bI[s2] == 0 && bJ[s2] == 0) factor_diag(s2, 0);
        for (int kb = 0; kb < nq; ++kb) {
            const int k0 = 4 * kb;
            __syncthreads();                  // R_kk and its inverse diagonal are published
            // block row kb: R_kb,j = R_kk^-T A_kb,j (forward substitution over its four rows)
#pragma unroll
            for (int s2 = 0; s2 < 2; ++s2) {
                if (bI[s2] != kb || bJ[s2] == kb) continue;
                float rdk[4][4], rr[4][4], ri[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float4 t = (k0 + c < m) ? *reinterpret_cast<const float4*>(A + (k0 + c) * lda + k0)
                                                  : make_float4(0.f, 0.f, 0.f, 0.f);
                    rdk[c][0] = t.x; rdk[c][1] = t.y; rdk[c][2] = t.z; rdk[c][3] = t.w;
                    ri[c] = sh_rinv[c];
                }
#pragma unroll
                for (int c = 0; c < 4; ++c)
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        float val = a[s2][c][v];
#pragma unroll
                        for (int l = 0; l < c; ++l) val = __fmaf_rn(-rdk[l][c], rr[l][v], val);
                        rr[c][v] = val * ri[c];
                    }
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (k0 + c < m) *reinterpret_cast<float4*>(A + (k0 + c) * lda + 4 * bJ[s2]) =
                                        make_float4(rr[c][0], rr[c][1], rr[c][2], rr[c][3]);
            }
            __syncthreads();                  // block row kb of R is published
            // rank-4 update of the blocks below block row kb, then the next diagonal block
#pragma unroll
            for (int s2 = 0; s2 < 2; ++s2) {
                if (bI[s2] <= kb) continue;
                float ri[4][4], rj[4][4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const bool live = k0 + c < m;
                    const float4 x = live ? *reinterpret_cast<const float4*>(A + (k0 + c) * lda + 4 * bI[s2])
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float4 y = live ? *reinterpret_cast<const float4*>(A + (k0 + c) * lda + 4 * bJ[s2])
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
                    ri[c][0] = x.x; ri[c][1] = x.y; ri[c][2] = x.z; ri[c][3] = x.w;
                    rj[c][0] = y.x; rj[c][1] = y.y; rj[c][2] = y.z; rj[c][3] = y.w;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        float acc = a[s2][u][v];
#pragma unroll
                        for (int c = 0; c < 4; ++c) acc = __fmaf_rn(-ri[c][u], rj[c][v], acc);
                        a[s2][u][v] = acc;
                    }
                if (bI[s2] == kb + 1 && bJ[s2] == kb + 1) factor_diag(s2, kb + 1);
            }
        }
    }
    // diagonal blocks of W = R^-1: warp p inverts R_pp, lane j solving for its
    // column by back substitution (W_lj = 0 below the diagonal, so every lane
    // runs the same loops)
    for (int p = warp; p < nb; p += nw) {
        const int p0 = p * kCB, bw = min(kCB, m - p0);
        const int jl = lane;
        if (jl < bw) W[(p0 + jl) * lda + p0 + jl] = __frcp_rn(A[(p0 + jl) * lda + p0 + jl]);
        for (int ii = bw - 2; ii >= 0; --ii) {
            float sacc = 0.f;
            for (int l = ii + 1; l < bw; ++l)
                sacc = __fmaf_rn(A[(p0 + ii) * lda + p0 + l], jl < bw ? W[(p0 + l) * lda + p0 + jl] : 0.f, sacc);
            if (jl < bw && jl > ii) W[(p0 + ii) * lda + p0 + jl] = -sacc / A[(p0 + ii) * lda + p0 + ii];
        }
    }
    __syncthreads();
    // off-diagonal blocks of W, one block diagonal sd = q - p at a time; thread = (pair, row i, column quad)
    for (int sd = 1; sd < nb; ++sd) {
        const int npairs = nb - sd;
        for (int e = tid; e < npairs * kCB * (kCB / 4); e += kCBThreads) {
            const int p = e / (kCB * kCB / 4), r = e % (kCB * kCB / 4), i = r / (kCB / 4), j = (r % (kCB / 4)) * 4;
            const int p0 = p * kCB, q0 = (p + sd) * kCB;
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            if (p0 + i < m && q0 + j < m) {
                const int cend = min(m, q0 + j + 4);
                for (int c = p0 + kCB; c < cend; ++c) {
                    const float rv = A[(p0 + i) * lda + c];
                    const float4 w4 = *reinterpret_cast<const float4*>(W + c * lda + q0 + j);
                    acc.x = __fmaf_rn(rv, w4.x, acc.x);
                    acc.y = __fmaf_rn(rv, w4.y, acc.y);
                    acc.z = __fmaf_rn(rv, w4.z, acc.z);
                    acc.w = __fmaf_rn(rv, w4.w, acc.w);
                }
            }
            *reinterpret_cast<float4*>(T + p * kCB * kCB + i * kCB + j) = acc;
        }
        __syncthreads();
        for (int e = tid; e < npairs * kCB * (kCB / 4); e += kCBThreads) {
            const int p = e / (kCB * kCB / 4), r = e % (kCB * kCB / 4), i = r / (kCB / 4), j = (r % (kCB / 4)) * 4;
            const int p0 = p * kCB, q0 = (p + sd) * kCB;
            if (p0 + i >= m || q0 + j >= m) continue;
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int c = i; c < kCB; ++c) {
                const float wv = W[(p0 + i) * lda + p0 + c];
                const float4 t4 = *reinterpret_cast<const float4*>(T + p * kCB * kCB + c * kCB + j);
                acc.x = __fmaf_rn(-wv, t4.x, acc.x);
                acc.y = __fmaf_rn(-wv, t4.y, acc.y);
                acc.z = __fmaf_rn(-wv, t4.z, acc.z);
                acc.w = __fmaf_rn(-wv, t4.w, acc.w);
            }
            *reinterpret_cast<float4*>(W + (p0 + i) * lda + q0 + j) = acc;
        }
        __syncthreads();
    }
    // kappa bound, then Rinv = D W
    {
        float wf = 0.f;
        for (int e = tid; e < m * lda; e += kCBThreads) wf = __fmaf_rn(W[e], W[e], wf);
        for (int o = 16; o > 0; o >>= 1) wf += __shfl_xor_sync(full, wf, o);
        if (lane == 0) red[warp] = wf;
        __syncthreads();
        if (tid == 0) {
            float t = 0.f;
            for (int w = 0; w < nw; ++w) t += red[w];
            const bool reject = bad || !(rowsum_max * t <= kCholKappaMax);
            if (fallback) *fallback = reject ? 1 : 0;
            else if (bad) set_status(status, kDevCholeskyBreakdown);
            if (next) *next = (reject || !(rowsum_max * t <= kCholSkipMax)) ? 1 : 0;
        }
    }
    for (int i = warp; i < m; i += nw) {
        const float di = dsc[i];
        for (int j = lane; j < m; j += 32) Rinv[i * m + j] = di * W[i * lda + j];
    }
}

// run_if (may be NULL): when *run_if == 0 the pass is skipped and Rinv = I, so
// that the following Q = V Rinv is an exact copy.  next: see kCholSkipMax.
__global__ void __launch_bounds__(kCBThreads, 1) chol_blocked_kernel(const float* __restrict__ Gf, int m,
                                                                   float* __restrict__ Rinv, int* fallback,
                                                                   int* status, int near_identity,
                                                                   const int* run_if, int* next) {
    if (run_if && *run_if == 0) {
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) Rinv[e] = (e / m == e % m) ? 1.f : 0.f;
        return;
    }
    chol_blocked_body(Gf, m, Rinv, fallback, status, near_identity, next);
}

// Q = V X with X = R^-1 upper triangular (row-major).  A block stages X and
// 32 rows of V in shared memory; thread (c, h) computes output column c for
// the 16 rows of half h: Q[r, c] = sum_{l <= c} V[r, l] X[l, c], V's rows
// read as float4 broadcasts.  The V block starts at a float offset rounded up
// to a multiple of 4 (16-byte aligned for any m).  Q must not alias V.
constexpr int kApplyRows = 32;
constexpr int kApplyHalf = kApplyRows / 2;

__host__ __device__ inline int apply_xs_floats(int m) { return (m * m + 3) & ~3; }

// Qb (may be NULL): Q's BF16 rounding as well, column c at Qb + c * ldb.
__device__ __forceinline__ void apply_rinv_body(const float* __restrict__ V, const float* __restrict__ Rinv,
                                                int64_t d, int m, float* __restrict__ Q, int block,
                                                __nv_bfloat16* __restrict__ Qb = nullptr, int64_t ldb = 0) {
    extern __shared__ __align__(16) float ars[];
    float* xs = ars;                          // m x m, X row-major
    float* vs = ars + apply_xs_floats(m);     // m x kApplyRows, vs[l][r] = V[r0 + r, l]
    const int64_t r0 = (int64_t)block * kApplyRows;
    const int mm = m * m, mm4 = mm / 4;
    if ((reinterpret_cast<uintptr_t>(Rinv) & 15) == 0) {
        const float4* x4 = reinterpret_cast<const float4*>(Rinv);
        for (int e = threadIdx.x; e < mm4; e += blockDim.x) reinterpret_cast<float4*>(xs)[e] = x4[e];
        for (int e = 4 * mm4 + threadIdx.x; e < mm; e += blockDim.x) xs[e] = Rinv[e];
    } else {
        for (int e = threadIdx.x; e < mm; e += blockDim.x) xs[e] = Rinv[e];
    }
    for (int e = threadIdx.x; e < m * kApplyRows; e += blockDim.x) {
        const int l = e / kApplyRows, r = e % kApplyRows;
        vs[e] = (r0 + r < d) ? V[(int64_t)l * d + r0 + r] : 0.f;
    }
    __syncthreads();
    const int mp = blockDim.x / 2;
    const int c = threadIdx.x % mp, h = threadIdx.x / mp;
    if (c >= m) return;
    float acc[kApplyHalf];
#pragma unroll
    for (int r = 0; r < kApplyHalf; ++r) acc[r] = 0.f;
    for (int l = 0; l <= c; ++l) {
        const float x = xs[l * m + c];
        const float4* v4 = reinterpret_cast<const float4*>(vs + l * kApplyRows + h * kApplyHalf);
#pragma unroll
        for (int q = 0; q < kApplyHalf / 4; ++q) {
            const float4 v = v4[q];
            acc[4 * q + 0] = __fmaf_rn(v.x, x, acc[4 * q + 0]);
            acc[4 * q + 1] = __fmaf_rn(v.y, x, acc[4 * q + 1]);
            acc[4 * q + 2] = __fmaf_rn(v.z, x, acc[4 * q + 2]);
            acc[4 * q + 3] = __fmaf_rn(v.w, x, acc[4 * q + 3]);
        }
    }
    const int64_t rb = r0 + h * kApplyHalf;
    float* out = Q + (int64_t)c * d + rb;
#pragma unroll
    for (int r = 0; r < kApplyHalf; ++r)
        if (rb + r < d) out[r] = acc[r];
    if (Qb) {
        __nv_bfloat16* ob = Qb + (int64_t)c * ldb + rb;
#pragma unroll
        for (int r = 0; r < kApplyHalf; ++r)
            if (rb + r < d) ob[r] = __float2bfloat16_rn(acc[r]);
    }
}

__global__ void __launch_bounds__(256) apply_rinv_kernel(const float* __restrict__ V, const float* __restrict__ Rinv,
                                                         int64_t d, int m, float* __restrict__ Q) {
    apply_rinv_body(V, Rinv, d, m, Q, blockIdx.x);
}

// ------------------------------------------------------------------ Jacobi

// Parallel-order (round-robin) two-sided Jacobi in FP32 on N = m rounded up to
// even; the extra index is a decoupled zero row/column.  Each step applies the
// N/2 disjoint rotations J of one round-robin round: A <- J^T A J, U <- U J.
// Warp w owns the pairs t = w, w + NW, ... of every step: its lanes compute
// those rotations (classical angle) in registers and broadcast them by
// shuffles, the warp rotates rows p, q of its pairs, and after a barrier
// columns p, q of A and U -- two barriers per step, every lane with several
// independent shared-memory accesses in flight.  The pairs of a step are
// disjoint, so the row pass of one warp never touches the rows whose
// entries another warp reads for its angles.  A rotation of pair (p, q) is
// skipped when |a_pq| <= tol * sqrt(|a_pp a_qq|), the relative criterion that
// keeps small eigenvalues accurate.  NT = 32 runs the whole solve in one warp
// (N <= 32).
constexpr int kJacobiMaxSweeps = 40;

__device__ __forceinline__ int rr_player(int pos, int step, int N) {
    if (pos == 0) return 0;
    int x = pos - 1 + step;              // < 2 (N - 1)
    if (x >= N - 1) x -= N - 1;
    return x + 1;
}

template <int NT>
__device__ __forceinline__ void jbar() {
    if (NT == 32) __syncwarp(); else __syncthreads();
}

template <int NT>
__device__ __forceinline__ void jacobi_f32_body(const double* __restrict__ G, int m, float* __restrict__ evals,
                                                float* __restrict__ Uf, int* sweeps_out, int* status) {
    constexpr int NW = NT / 32;
    constexpr int NMAX = NT == 32 ? 32 : kMaxM;           // largest N this instance runs
    constexpr int KP = (NMAX / 2 + NW - 1) / NW;          // pairs per warp and step
    constexpr int RPL = NMAX / 32;                        // row / column entries per lane
    static_assert(KP <= 32, "one lane per owned pair");
    extern __shared__ float js[];
    const int N = m + (m & 1);
    const int H = N / 2;
    const int S = N + 1;            // padded row stride: row and column passes are bank-conflict free
    float* A = js;                  // N x S
    float* U = A + N * S;           // N x S (column j = eigenvector j)
    __shared__ int rotated;
    const unsigned full = 0xffffffffu;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    for (int e = threadIdx.x; e < N * N; e += NT) {
        const int i = e / N, j = e % N;
        A[i * S + j] = (i < m && j < m) ? (float)(0.5 * (G[i * m + j] + G[j * m + i])) : 0.f;
        U[i * S + j] = (i == j) ? 1.f : 0.f;
    }
    jbar<NT>();
    const float tol = 4.0f * 5.96e-8f;
    int sweep = 0;
    for (; sweep < kJacobiMaxSweeps; ++sweep) {
        if (threadIdx.x == 0) rotated = 0;
        jbar<NT>();
        for (int step = 0; step < N - 1; ++step) {
            // rotation of the pair t = warp + lane * NW (lanes < KP)
            int myp = 0, myq = 0;
            float myc = 1.f, mys = 0.f, mydp = 0.f, mydq = 0.f;
            {
                const int t = warp + lane * NW;
                if (lane < KP && t < H) {
                    int p = rr_player(t, step, N), q = rr_player(N - 1 - t, step, N);
                    if (p > q) { const int x = p; p = q; q = x; }
                    myp = p;
                    myq = q;
                    const float apq = A[p * S + q], app = A[p * S + p], aqq = A[q * S + q];
                    float tt = 0.f;
                    if (fabsf(apq) > 1e-30f && fabsf(apq) > tol * sqrtf(fabsf(app)) * sqrtf(fabsf(aqq))) {
                        const float tau = (aqq - app) / (2.0f * apq);
                        if (fabsf(tau) > 1e18f) {
                            tt = 0.5f / tau;
                        } else {
                            tt = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.0f + tau * tau));
                        }
                        myc = 1.0f / sqrtf(1.0f + tt * tt);
                        mys = tt * myc;
                        rotated = 1;
                    }
                    mydp = app - tt * apq;
                    mydq = aqq + tt * apq;
                }
            }
            // rows p, q: A <- J^T A
#pragma unroll
            for (int k = 0; k < KP; ++k) {
                if (warp + k * NW >= H) break;
                const float s = __shfl_sync(full, mys, k);
                const float c = __shfl_sync(full, myc, k);
                const int p = __shfl_sync(full, myp, k), q = __shfl_sync(full, myq, k);
                if (s == 0.f) continue;
                float ap[RPL], aq[RPL];
#pragma unroll
                for (int r = 0; r < RPL; ++r) {
                    const int j = lane + 32 * r;
                    ap[r] = j < N ? A[p * S + j] : 0.f;
                    aq[r] = j < N ? A[q * S + j] : 0.f;
                }
#pragma unroll
                for (int r = 0; r < RPL; ++r) {
                    const int j = lane + 32 * r;
                    if (j < N) {
                        A[p * S + j] = c * ap[r] - s * aq[r];
                        A[q * S + j] = s * ap[r] + c * aq[r];
                    }
                }
            }
            jbar<NT>();
            // columns p, q: A <- A J, U <- U J; the pair's own 2x2 block gets the
            // exact zero and the tangent-formula diagonal
#pragma unroll
            for (int k = 0; k < KP; ++k) {
                if (warp + k * NW >= H) break;
                const float s = __shfl_sync(full, mys, k);
                const float c = __shfl_sync(full, myc, k);
                const int p = __shfl_sync(full, myp, k), q = __shfl_sync(full, myq, k);
                const float dp = __shfl_sync(full, mydp, k), dq = __shfl_sync(full, mydq, k);
                if (s == 0.f) continue;
                float aip[RPL], aiq[RPL], uip[RPL], uiq[RPL];
#pragma unroll
                for (int r = 0; r < RPL; ++r) {
                    const int i = lane + 32 * r;
                    const bool in = i < N;
                    aip[r] = in ? A[i * S + p] : 0.f;
                    aiq[r] = in ? A[i * S + q] : 0.f;
                    uip[r] = in ? U[i * S + p] : 0.f;
                    uiq[r] = in ? U[i * S + q] : 0.f;
                }
#pragma unroll
                for (int r = 0; r < RPL; ++r) {
                    const int i = lane + 32 * r;
                    if (i >= N) continue;
                    if (i == p) {
                        A[p * S + p] = dp;
                        A[p * S + q] = 0.f;
                    } else if (i == q) {
                        A[q * S + p] = 0.f;
                        A[q * S + q] = dq;
                    } else {
                        A[i * S + p] = c * aip[r] - s * aiq[r];
                        A[i * S + q] = s * aip[r] + c * aiq[r];
                    }
                    U[i * S + p] = c * uip[r] - s * uiq[r];
                    U[i * S + q] = s * uip[r] + c * uiq[r];
                }
            }
            jbar<NT>();
        }
        const int any = rotated;
        jbar<NT>();
        if (!any) break;
    }
    if (threadIdx.x == 0) {
        if (sweep >= kJacobiMaxSweeps) set_status(status, kDevJacobiNoConverge);
        *sweeps_out = sweep;
    }
    for (int e = threadIdx.x; e < m * m; e += NT) {
        const int i = e / m, j = e % m;
        Uf[j * m + i] = U[i * S + j];      // column-major m x m
    }
    for (int i = threadIdx.x; i < m; i += NT) evals[i] = A[i * S + i];
}

template <int NT>
__global__ void __launch_bounds__(NT) jacobi_f32_kernel(const double* __restrict__ G, int m, float* __restrict__ evals,
                                                        float* __restrict__ Uf, int* sweeps_out, int* status) {
    jacobi_f32_body<NT>(G, m, evals, Uf, sweeps_out, status);
}

// FP64 polish: u_j <- u_j / |u_j|, lambda_j = u_j^T G u_j (Rayleigh quotient).
__device__ __forceinline__ void rayleigh_f64_body(const double* __restrict__ G, int m, const float* __restrict__ Uf,
                                                  double* __restrict__ U64, double* __restrict__ lam, int j) {
    __shared__ double u[kMaxM];
    __shared__ double red[32];
    for (int i = threadIdx.x; i < m; i += blockDim.x) u[i] = (double)Uf[j * m + i];
    __syncthreads();
    double nrm = 0.0, rq = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double gi = 0.0;
        for (int l = 0; l < m; ++l) gi += 0.5 * (G[i * m + l] + G[l * m + i]) * u[l];
        rq += u[i] * gi;
        nrm += u[i] * u[i];
    }
    // block reduce (two values)
    for (int o = 16; o > 0; o >>= 1) {
        rq += __shfl_down_sync(0xffffffff, rq, o);
        nrm += __shfl_down_sync(0xffffffff, nrm, o);
    }
    const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
    __shared__ double red2[32];
    if (lane == 0) { red[w] = rq; red2[w] = nrm; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) { a += red[i]; b += red2[i]; }
        red[0] = a;
        red2[0] = b;
    }
    __syncthreads();
    const double n2 = red2[0];
    const double inv = n2 > 0.0 ? 1.0 / sqrt(n2) : 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) U64[j * m + i] = u[i] * inv;
    if (threadIdx.x == 0) lam[j] = n2 > 0.0 ? red[0] / n2 : 0.0;
}

__global__ void rayleigh_f64_kernel(const double* __restrict__ G, int m, const float* __restrict__ Uf,
                                    double* __restrict__ U64, double* __restrict__ lam) {
    rayleigh_f64_body(G, m, Uf, U64, lam, blockIdx.x);
}

// Sort eigenpairs descending (stable in the index), in one CTA.
__device__ __forceinline__ void sort_desc_body(const double* __restrict__ lam, const double* __restrict__ U64, int m,
                                               double* __restrict__ w, double* __restrict__ U) {
    __shared__ int rank[kMaxM];
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        int r = 0;
        const double lj = lam[j];
        for (int i = 0; i < m; ++i) {
            const double li = lam[i];
            r += (li > lj) || (li == lj && i < j);
        }
        rank[j] = r;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < m; j += blockDim.x) w[rank[j]] = lam[j];
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int j = e / m, i = e % m;
        U[rank[j] * m + i] = U64[j * m + i];
    }
}

__global__ void sort_desc_kernel(const double* __restrict__ lam, const double* __restrict__ U64, int m,
                                 double* __restrict__ w, double* __restrict__ U) {
    sort_desc_body(lam, U64, m, w, U);
}

// ------------------------------------------------------------------ rotate + sign

__device__ __forceinline__ void rotate_body(const float* __restrict__ Q, int64_t d, int m,
                                            const double* __restrict__ U, float* __restrict__ E, int bx, int j) {
    __shared__ float u[kMaxM];
    for (int i = threadIdx.x; i < m; i += blockDim.x) u[i] = (float)U[j * m + i];
    __syncthreads();
    const int64_t r = (int64_t)bx * blockDim.x + threadIdx.x;
    if (r >= d) return;
    float s = 0.f;
    for (int i = 0; i < m; ++i) s = __fmaf_rn(Q[(int64_t)i * d + r], u[i], s);
    E[(int64_t)j * d + r] = s;
}

__global__ void rotate_kernel(const float* __restrict__ Q, int64_t d, int m, const double* __restrict__ U, int k,
                              float* __restrict__ E) {
    (void)k;
    rotate_body(Q, d, m, U, E, blockIdx.x, blockIdx.y);
}

__device__ __forceinline__ void sign_body(float* __restrict__ E, int64_t d, const double* __restrict__ w,
                                          double inv_n, double* __restrict__ lambda, int j) {
    float* e = E + (int64_t)j * d;
    float best = -1.f;
    int64_t bi = 0;
    for (int64_t r = threadIdx.x; r < d; r += blockDim.x) {
        const float a = fabsf(e[r]);
        if (a > best) { best = a; bi = r; }     // increasing r: first maximum kept
    }
    __shared__ float sb[1024];
    __shared__ long long si[1024];
    sb[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            const float b2 = sb[threadIdx.x + o];
            const long long i2 = si[threadIdx.x + o];
            if (b2 > sb[threadIdx.x] || (b2 == sb[threadIdx.x] && i2 < si[threadIdx.x])) {
                sb[threadIdx.x] = b2;
                si[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    const bool flip = e[si[0]] < 0.f;
    __syncthreads();
    if (flip)
        for (int64_t r = threadIdx.x; r < d; r += blockDim.x) e[r] = -e[r];
    if (threadIdx.x == 0) lambda[j] = w[j] * inv_n;
}

__global__ void sign_kernel(float* __restrict__ E, int64_t d, const double* __restrict__ w, double inv_n,
                            double* __restrict__ lambda) {
    sign_body(E, d, w, inv_n, lambda, blockIdx.x);
}

// ------------------------------------------------------------------ Oja / Sanger


// W[r][j] += c (Z[r][j] - sum_{l <= j} W[r][l] S[l][j]) with S = Y^T Y: one thread per
// (row, column), kOjaRows rows of W and S (as FP32) staged in shared memory per CTA.
constexpr int kOjaRows = 8;
__global__ void oja_update_kernel(float* __restrict__ W, const float* __restrict__ Z, const double* __restrict__ S,
                                  int64_t d, int m, float c_host, const float* __restrict__ c_dev) {
    const float c = c_dev ? *c_dev : c_host;
    extern __shared__ float sm[];
    const int ws = m + 1;                  // row stride: consecutive rows in different banks
    float* Ss = sm;                        // m x m (row-major)
    float* w = sm + m * m;                 // kOjaRows x ws, the old rows of W
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) Ss[e] = (float)S[e];
    const int64_t r0 = (int64_t)blockIdx.x * kOjaRows;
    for (int e = threadIdx.x; e < kOjaRows * m; e += blockDim.x) {
        const int i = e % kOjaRows, j = e / kOjaRows;      // consecutive threads: consecutive rows
        w[i * ws + j] = r0 + i < d ? W[(int64_t)j * d + r0 + i] : 0.f;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kOjaRows * m; e += blockDim.x) {
        const int i = e % kOjaRows, j = e / kOjaRows;      // consecutive threads: consecutive rows (coalesced)
        const int64_t r = r0 + i;
        if (r >= d) continue;
        const float* wr = w + i * ws;
        float acc = 0.f;
        for (int l = 0; l <= j; ++l) acc = __fmaf_rn(wr[l], Ss[l * m + j], acc);
        W[(int64_t)j * d + r] = wr[j] + c * (Z[(int64_t)j * d + r] - acc);
    }
}

// Step state of graph-replayed minibatch steps: step t's batch starts at row
// (t mod per_epoch) b, and Oja's coefficient is lr / (t + lr_offset) / b, both
// computed here in the same double arithmetic as the host's; then t advances.
__global__ void primer_step_kernel(PrimerStep* ps, int64_t per_epoch, int64_t b, double lr, double lr_offset) {
    const int64_t t = ps->t;
    ps->row0 = (t % per_epoch) * b;
    ps->c = (float)(lr / ((double)t + lr_offset) / (double)b);
    ps->t = t + 1;
}

__global__ void primer_set_kernel(PrimerStep* ps, int64_t t) { ps->t = t; }

// ------------------------------------------------------------------ EigenGame

// coef[i][j] = C_ij / C_ii (i < j), alpha_j = 2 C_jj - 2 sum_{i<j} C_ij^2 / C_ii, C scaled by 1/b.
// One block per column j: thread i forms the term of player i, the block sums alpha_j (FP64).
constexpr int kCoefThreads = 128;
__global__ void eg_coef_kernel(const double* __restrict__ C, int m, double inv_b, float* __restrict__ coef,
                               float* __restrict__ alpha) {
    __shared__ double red[kCoefThreads / 32];
    const int j = blockIdx.x;
    double part = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const double cii = C[i * m + i] * inv_b;
        const double cij = 0.5 * (C[i * m + j] + C[j * m + i]) * inv_b;
        const bool use = i < j && cii != 0.0;
        const double q = use ? cij / cii : 0.0;
        coef[i * m + j] = (float)q;
        if (use) part += cij * q;
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int w = 0; w < kCoefThreads / 32; ++w) sum += red[w];
        alpha[j] = (float)(2.0 * C[j * m + j] * inv_b - 2.0 * sum);
    }
}

// One EigenGame step for `rows` rows of V per CTA, one thread per (row, player):
// g_j = 2 (Z_j / b) - 2 sum_{i<j} coef_ij (Z_i / b) - alpha_j v_j (the utility gradient
// with the Riemannian projection folded into alpha), Nesterov: buf <- mu buf + g,
// v <- v + lr (mu buf + g); then each column's squared norm over the CTA's rows as a
// double-float partial (colpart[block][j]).
// (16 rows per CTA for short bases, 64 for tall ones, where the m x m coefficients
// every CTA stages would otherwise dominate the traffic.)
inline int eg_rows_per_block(int64_t d) { return d >= 65536 ? 64 : 16; }

__global__ void eg_step_kernel(float* __restrict__ V, float* __restrict__ buf, const float* __restrict__ Z,
                               const float* __restrict__ coef_g, const float* __restrict__ alpha_g, int64_t d, int m,
                               int rows, float inv_b, float lr, float mu, float2* __restrict__ colpart) {
    extern __shared__ float sm[];
    // row stride m + 1: a warp's threads take consecutive rows, which a stride
    // of m (a multiple of 32) would put in one shared-memory bank
    const int ms = m + 1;
    float* coef = sm;                      // m x m
    float* alpha = coef + m * m;           // m
    float* mv = alpha + m;                 // rows x ms: Z rows / b
    float* vn = mv + rows * ms;            // rows x ms: the new rows of V
    const int64_t r0 = (int64_t)blockIdx.x * rows;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) coef[e] = coef_g[e];
    for (int e = threadIdx.x; e < m; e += blockDim.x) alpha[e] = alpha_g[e];
    for (int e = threadIdx.x; e < rows * m; e += blockDim.x) {
        const int i = e % rows, j = e / rows;      // consecutive threads: consecutive rows
        mv[i * ms + j] = r0 + i < d ? Z[(int64_t)j * d + r0 + i] * inv_b : 0.f;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < rows * m; e += blockDim.x) {
        const int i = e % rows, j = e / rows;
        const int64_t r = r0 + i;
        float out = 0.f;
        if (r < d) {
            const float* mr = mv + i * ms;
            float g = 2.f * mr[j];
            for (int l = 0; l < j; ++l) g = __fmaf_rn(-2.f * coef[l * m + j], mr[l], g);
            const float v = V[(int64_t)j * d + r];
            g = __fmaf_rn(-alpha[j], v, g);                       // Riemannian projection
            const float b = __fmaf_rn(mu, buf[(int64_t)j * d + r], g);
            buf[(int64_t)j * d + r] = b;
            out = __fmaf_rn(lr, __fmaf_rn(mu, b, g), v);          // Nesterov step
            V[(int64_t)j * d + r] = out;
        }
        vn[i * ms + j] = out;
    }
    __syncthreads();
    // this block's part of each column's squared norm (squares exact as hi + lo)
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        dfloat q = {0.f, 0.f};
        for (int i = 0; i < rows; ++i) {
            const float x = vn[i * ms + j];
            const float p = __fmul_rn(x, x);
            q = df_addx(q, df_norm(p, __fmaf_rn(x, x, -p)));
        }
        colpart[(int64_t)blockIdx.x * m + j] = make_float2(q.hi, q.lo);
    }
}

// One block per column: thread t adds blocks t, t + blockDim, ... in order,
// then a fixed tree in shared memory; the column's scale 1/norm is written as
// a pair of floats (hi, lo) with hi + lo = 1/norm to about 2^-48.
constexpr int kNormThreads = 256;
__global__ void colnorm_reduce_kernel(const float2* __restrict__ colpart, int nblk, int m, float2* __restrict__ inv) {
    __shared__ float2 s[kNormThreads];
    const int j = blockIdx.x, t = threadIdx.x;
    dfloat q = {0.f, 0.f};
    for (int b = t; b < nblk; b += kNormThreads) {
        const float2 o = colpart[(int64_t)b * m + j];
        q = df_addx(q, df_norm(o.x, o.y));
    }
    s[t] = make_float2(q.hi, q.lo);
    __syncthreads();
    for (int h = kNormThreads / 2; h > 0; h >>= 1) {
        if (t < h) {
            q = df_addx(df_norm(s[t].x, s[t].y), df_norm(s[t + h].x, s[t + h].y));
            s[t] = make_float2(q.hi, q.lo);
        }
        __syncthreads();
    }
    if (t == 0) {
        const double n2 = (double)s[0].x + (double)s[0].y;
        const double r = n2 > 0.0 ? 1.0 / sqrt(n2) : 0.0;
        const float hi = (float)r;
        inv[j] = make_float2(hi, (float)(r - (double)hi));
    }
}

// V[:, j] *= 1/norm_j: the product with the pair (hi, lo) rounded once (the
// FMA gives v*hi's exact error; v*lo and that error are added before rounding).
__global__ void colscale_kernel(float* __restrict__ V, int64_t d, const float2* __restrict__ inv) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= d) return;
    const float2 s = inv[blockIdx.y];
    float* v = V + (int64_t)blockIdx.y * d + r;
    const float x = *v;
    const float p = __fmul_rn(x, s.x);
    *v = __fadd_rn(p, __fmaf_rn(x, s.y, __fmaf_rn(x, s.x, -p)));
}

// ------------------------------------------------------------------ Philox + Box-Muller

struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox_round(U4 c, uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t lo0 = M0 * c.x, hi0 = __umulhi(M0, c.x);
    const uint32_t lo1 = M1 * c.z, hi1 = __umulhi(M1, c.z);
    U4 o;
    o.x = hi1 ^ c.y ^ k0;
    o.y = lo1;
    o.z = hi0 ^ c.w ^ k1;
    o.w = lo0;
    return o;
}

// Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11).
__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    c = philox_round(c, k0, k1);
#pragma unroll
    for (int i = 1; i < 10; ++i) {
        k0 += W0;
        k1 += W1;
        c = philox_round(c, k0, k1);
    }
    return c;
}

__global__ void init_gaussian_kernel(float* __restrict__ V, int64_t count, uint64_t seed) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g * 4 >= count) return;
    U4 c{(uint32_t)g, (uint32_t)(g >> 32), 0u, 0u};
    const U4 o = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    const float inv32 = 2.3283064365386963e-10f;   // 2^-32
    const float u1 = ((float)o.x + 1.0f) * inv32, u2 = (float)o.y * inv32;
    const float u3 = ((float)o.z + 1.0f) * inv32, u4 = (float)o.w * inv32;
    const float r1 = sqrtf(-2.0f * logf(fminf(u1, 1.0f))), r2 = sqrtf(-2.0f * logf(fminf(u3, 1.0f)));
    float s1, c1, s2, c2;
    sincospif(2.0f * u2, &s1, &c1);
    sincospif(2.0f * u4, &s2, &c2);
    const float z[4] = {r1 * c1, r1 * s1, r2 * c2, r2 * s2};
    for (int i = 0; i < 4; ++i)
        if (g * 4 + i < count) V[g * 4 + i] = z[i];
}

// ------------------------------------------------------------------ quantisers

__global__ void quantize_bf16_kernel(const float* __restrict__ X, int64_t n, int64_t d, int64_t ld_in,
                                     uint16_t* __restrict__ out, int64_t ld_out) {
    const int64_t r = blockIdx.y;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < d; j += (int64_t)gridDim.x * blockDim.x) {
        const __nv_bfloat16 b = __float2bfloat16_rn(X[r * ld_in + j]);
        out[r * ld_out + j] = *reinterpret_cast<const uint16_t*>(&b);
    }
}

// Eight values per thread (two 16-byte loads, one 16-byte store) over the whole
// matrix as one flat index, for rows whose pitches keep every group of eight aligned.
__global__ void quantize_bf16_vec8_kernel(const float* __restrict__ X, int64_t n, int64_t d, int64_t ld_in,
                                          uint16_t* __restrict__ out, int64_t ld_out) {
    const int64_t per_row = d / 8, total = n * per_row;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / per_row, j = (e - r * per_row) * 8;
        const float4 a = __ldcs(reinterpret_cast<const float4*>(X + r * ld_in + j));
        const float4 b = __ldcs(reinterpret_cast<const float4*>(X + r * ld_in + j + 4));
        __nv_bfloat162 p0 = __floats2bfloat162_rn(a.x, a.y), p1 = __floats2bfloat162_rn(a.z, a.w);
        __nv_bfloat162 p2 = __floats2bfloat162_rn(b.x, b.y), p3 = __floats2bfloat162_rn(b.z, b.w);
        uint4 o;
        o.x = *reinterpret_cast<uint32_t*>(&p0);
        o.y = *reinterpret_cast<uint32_t*>(&p1);
        o.z = *reinterpret_cast<uint32_t*>(&p2);
        o.w = *reinterpret_cast<uint32_t*>(&p3);
        *reinterpret_cast<uint4*>(out + r * ld_out + j) = o;
    }
}

__global__ void quantize_fp8_kernel(const float* __restrict__ X, int64_t d, int64_t ld_in, uint8_t* __restrict__ out,
                                    int64_t ld_out, float* __restrict__ scales) {
    const int64_t r = blockIdx.x;
    const float* x = X + r * ld_in;
    float amax = 0.f;
    for (int64_t j = threadIdx.x; j < d; j += blockDim.x) amax = fmaxf(amax, fabsf(x[j]));
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffff, amax, o));
    __shared__ float wm[32];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x / 32] = amax;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x + 31) / 32 ? wm[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffff, v, o));
        if (threadIdx.x == 0) wm[0] = v;
    }
    __syncthreads();
    amax = wm[0];
    const float s = amax > 0.f ? __fdiv_rn(amax, 448.0f) : 1.0f;
    if (threadIdx.x == 0) scales[r] = s;
    for (int64_t j = threadIdx.x; j < d; j += blockDim.x) {
        const float q = __fdiv_rn(x[j], s);
        out[r * ld_out + j] = (uint8_t)__nv_cvt_float_to_fp8(q, __NV_SATFINITE, __NV_E4M3);
    }
}

// One row per CTA of 256 threads held in registers (VPT float4 chunks a thread,
// d % 4 == 0, 16-byte aligned rows): one read of the row for both its maximum and
// its codes, four codes stored as one 32-bit word.
template <int VPT>
__global__ void __launch_bounds__(256) quantize_fp8_vec4_kernel(const float* __restrict__ X, int64_t d,
                                                                int64_t ld_in, uint8_t* __restrict__ out,
                                                                int64_t ld_out, float* __restrict__ scales) {
    const int64_t r = blockIdx.x;
    const float4* x = reinterpret_cast<const float4*>(X + r * ld_in);
    const int64_t chunks = d / 4;
    float4 v[VPT];
    float amax = 0.f;
#pragma unroll
    for (int i = 0; i < VPT; ++i) {
        const int64_t c = (int64_t)i * 256 + threadIdx.x;
        v[i] = c < chunks ? __ldcs(x + c) : make_float4(0.f, 0.f, 0.f, 0.f);
        amax = fmaxf(amax, fmaxf(fmaxf(fabsf(v[i].x), fabsf(v[i].y)), fmaxf(fabsf(v[i].z), fabsf(v[i].w))));
    }
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffff, amax, o));
    __shared__ float wm[8];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x / 32] = amax;
    __syncthreads();
    amax = wm[0];
#pragma unroll
    for (int w = 1; w < 8; ++w) amax = fmaxf(amax, wm[w]);
    const float s = amax > 0.f ? __fdiv_rn(amax, 448.0f) : 1.0f;
    if (threadIdx.x == 0) scales[r] = s;
    uint32_t* o = reinterpret_cast<uint32_t*>(out + r * ld_out);
#pragma unroll
    for (int i = 0; i < VPT; ++i) {
        const int64_t c = (int64_t)i * 256 + threadIdx.x;
        if (c >= chunks) break;
        const uint32_t q0 = __nv_cvt_float_to_fp8(__fdiv_rn(v[i].x, s), __NV_SATFINITE, __NV_E4M3);
        const uint32_t q1 = __nv_cvt_float_to_fp8(__fdiv_rn(v[i].y, s), __NV_SATFINITE, __NV_E4M3);
        const uint32_t q2 = __nv_cvt_float_to_fp8(__fdiv_rn(v[i].z, s), __NV_SATFINITE, __NV_E4M3);
        const uint32_t q3 = __nv_cvt_float_to_fp8(__fdiv_rn(v[i].w, s), __NV_SATFINITE, __NV_E4M3);
        o[c] = q0 | (q1 << 8) | (q2 << 16) | (q3 << 24);
    }
}

__global__ void copy_kernel(const float* __restrict__ s, float* __restrict__ d, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d[i] = s[i];
}

template <typename K>
cudaError_t allow_smem(K kernel, size_t bytes) {
    return smem_at_least(reinterpret_cast<const void*>(kernel), bytes);
}

// ------------------------------------------------------------------ grouped launches
//
// The same bodies over many instances at once (grouped.h): block b of the grid
// belongs to instance group_find(tab, b) and is its block b - tab.base[i].

__global__ void gram_df_grouped_kernel(const GInst* __restrict__ gi, GTable tab, int src, int gated) {
    const int i = group_find(tab, blockIdx.x);
    const GInst& g = gi[i];
    if (gated && *g.next == 0) return;                 // this instance's second pass is skipped
    const int local = blockIdx.x - tab.base[i], T = g.gram_T;
    const int ti = local % T, tj = (local / T) % T, p = local / (T * T);
    const float* A = garray(g, src);
    gram_df_body(A, A, g.d, g.m, g.gram_part, (g.d + g.gram_P - 1) / g.gram_P, ti, tj, p);
}

__global__ void gram_reduce_grouped_kernel(const GInst* __restrict__ gi, GTable tab, int gated) {
    const int i = group_find(tab, blockIdx.x);
    const GInst& g = gi[i];
    if (gated && *g.next == 0) return;
    gram_reduce_body(g.gram_part, g.gram_P, g.m, g.gram_L, true, g.G, g.Gf, blockIdx.x - tab.base[i]);
}

__global__ void __launch_bounds__(kCBThreads, 1) chol_blocked_grouped_kernel(const GInst* __restrict__ gi,
                                                                           int near_identity, int span_only,
                                                                           int gated) {
    const GInst& g = gi[blockIdx.x];
    if (gated && *g.next == 0) {
        for (int e = threadIdx.x; e < g.m * g.m; e += blockDim.x) g.Rinv[e] = (e / g.m == e % g.m) ? 1.f : 0.f;
        return;
    }
    chol_blocked_body(g.Gf, g.m, g.Rinv, near_identity ? nullptr : g.flag, g.status, near_identity,
                      span_only ? g.next : nullptr);
    if (!near_identity) {
        // a rejected FP32 factor is redone in double-float by the same block
        // (one launch instead of a second, mostly empty one)
        __syncthreads();
        if (*(volatile int*)g.flag) cholesky_body<true>(g.G, g.m, g.Rinv, g.status);
    }
}

// split: also write Q's BF16 rounding into Vp (the next pass's operand; its
// padding rows and columns stay zero from the set-up).
__global__ void __launch_bounds__(256) apply_rinv_grouped_kernel(const GInst* __restrict__ gi, GTable tab, int src,
                                                                 int dst, int split) {
    const int i = group_find(tab, blockIdx.x);
    const GInst& g = gi[i];
    apply_rinv_body(garray(g, src), g.Rinv, g.d, g.m, garray(g, dst), blockIdx.x - tab.base[i],
                    split ? g.Vp : nullptr, g.ldv);
}

// BF16 rounding of every instance's FP32 X (d % 8 == 0, 16-byte aligned rows), eight values a thread.
__global__ void quantize_bf16_grouped_kernel(const float* const* __restrict__ X32, const int64_t* __restrict__ ld32,
                                             const GInst* __restrict__ gi, GTable tab) {
    const int i = group_find(tab, blockIdx.x);
    const GInst& g = gi[i];
    const int64_t per_row = g.d / 8;
    const int64_t e = (int64_t)(blockIdx.x - tab.base[i]) * blockDim.x + threadIdx.x;
    if (e >= g.n * per_row) return;
    const int64_t r = e / per_row, j = (e - r * per_row) * 8;
    const float* x = X32[i] + r * ld32[i] + j;
    const float4 a = __ldcs(reinterpret_cast<const float4*>(x));
    const float4 b = __ldcs(reinterpret_cast<const float4*>(x + 4));
    __nv_bfloat162 p0 = __floats2bfloat162_rn(a.x, a.y), p1 = __floats2bfloat162_rn(a.z, a.w);
    __nv_bfloat162 p2 = __floats2bfloat162_rn(b.x, b.y), p3 = __floats2bfloat162_rn(b.z, b.w);
    uint4 o;
    o.x = *reinterpret_cast<uint32_t*>(&p0);
    o.y = *reinterpret_cast<uint32_t*>(&p1);
    o.z = *reinterpret_cast<uint32_t*>(&p2);
    o.w = *reinterpret_cast<uint32_t*>(&p3);
    *reinterpret_cast<uint4*>(const_cast<__nv_bfloat16*>(static_cast<const __nv_bfloat16*>(g.X)) + r * g.ld + j) = o;
}

// The pPCA step's eigensolve (Algorithm 1, step 4) per instance: Jacobi on
// block i, the FP64 Rayleigh polish on blocks (instance, eigenvector), the sort.
__global__ void __launch_bounds__(512) jacobi_grouped_kernel(const GInst* __restrict__ gi) {
    const GInst& g = gi[blockIdx.x];
    jacobi_f32_body<512>(g.Gp, g.m, g.evals, g.Uf, g.sweeps, g.status);
}

__global__ void rayleigh_grouped_kernel(const GInst* __restrict__ gi, GTable tab) {
    const int i = group_find(tab, blockIdx.x);
    const GInst& g = gi[i];
    rayleigh_f64_body(g.Gp, g.m, g.Uf, g.U64, g.lam, blockIdx.x - tab.base[i]);
}

__global__ void sort_grouped_kernel(const GInst* __restrict__ gi) {
    const GInst& g = gi[blockIdx.x];
    sort_desc_body(g.lam, g.U64, g.m, g.w, g.U);
}

// Step 5 per instance: E = Q U[:, :k] (Q = orth(V), held in Z), the sign
// convention and lambda = w / n.
__global__ void rotate_grouped_kernel(const GInst* __restrict__ gi, GTable tab) {
    const int i = group_find(tab, blockIdx.x);
    const GInst& g = gi[i];
    const int local = blockIdx.x - tab.base[i];
    const int nbx = (int)((g.d + blockDim.x - 1) / blockDim.x);
    rotate_body(g.Z, g.d, g.m, g.U, g.E, local % nbx, local / nbx);
}

__global__ void sign_grouped_kernel(const GInst* __restrict__ gi, GTable tab) {
    const int i = group_find(tab, blockIdx.x);
    const GInst& g = gi[i];
    sign_body(g.E, g.d, g.w, 1.0 / (double)g.n, g.lambda, blockIdx.x - tab.base[i]);
}

// The primed basis of every instance that asked for it.
__global__ void copy_vout_grouped_kernel(const GInst* __restrict__ gi, GTable tab) {
    const int i = group_find(tab, blockIdx.x);
    const GInst& g = gi[i];
    const int64_t e = (int64_t)(blockIdx.x - tab.base[i]) * blockDim.x + threadIdx.x;
    if (g.V_out && e < g.d * g.m) g.V_out[e] = g.V[e];
}

// Starting bases: V0 of every instance that has one, copied into its V.
__global__ void copy_v0_grouped_kernel(const GInst* __restrict__ gi, GTable tab) {
    const int i = group_find(tab, blockIdx.x);
    const GInst& g = gi[i];
    const int64_t e = (int64_t)(blockIdx.x - tab.base[i]) * blockDim.x + threadIdx.x;
    if (g.V0 && e < g.d * g.m) g.V[e] = g.V0[e];
}

}  // namespace

// ============================================================================ launchers

cudaError_t smem_at_least(const void* func, size_t bytes) {
    if (bytes <= 32 * 1024) return cudaSuccess;          // within every kernel's default limit
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> set;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    size_t& now = set[std::make_pair(dev, func)];
    if (bytes <= now) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) now = bytes;
    return e;
}

// The workspace sized for m also serves every narrower basis.
size_t gram_part_floats(int64_t d, int m) {
    size_t most = 0;
    for (int w = 1; w <= m; ++w) {
        const size_t f = (size_t)gram_nslices(d, w) * w * w * 2;
        most = f > most ? f : most;
    }
    return most;
}

cudaError_t gram_df(const float* A, const float* B, int64_t d, int m, double* G, float* part, cudaStream_t st,
                    float* Gf, const int* run_if) {
    const int P = gram_nslices(d, m);
    const int64_t slice = (d + P - 1) / P;
    const int T = (m + kGramTile - 1) / kGramTile;
    note_launch();
    gram_df_kernel<<<dim3(T, T, P), 256, 0, st>>>(A, B, d, m, part, slice, run_if);
    const int L = gram_reduce_lanes(P);
    note_launch();
    gram_reduce_kernel<<<ceil_div_i((int64_t)m * m * L, 256), 256, 0, st>>>(part, P, m, L, A == B, G, Gf, run_if);
    return cudaGetLastError();
}

cudaError_t cholesky_adaptive(double* G, const float* Gf, int m, float* Rinv, bool may_fall_back, int* flag,
                              int* status, cudaStream_t st, const float* Zdf, int64_t d, float* part, int* next,
                              const int* run_if) {
    const size_t lda = (size_t)((m + 3) & ~3);
    const size_t smem = ((size_t)2 * m * lda + (size_t)((m + kCB - 1) / kCB) * kCB * kCB + m) * sizeof(float);
    cudaError_t e = allow_smem(chol_blocked_kernel, smem);
    if (e != cudaSuccess) return e;
    note_launch();
    chol_blocked_kernel<<<1, kCBThreads, smem, st>>>(Gf, m, Rinv, may_fall_back ? flag : nullptr, status,
                                                      may_fall_back ? 0 : 1, run_if, next);
    e = cudaGetLastError();
    if (e != cudaSuccess || !may_fall_back) return e;
    if (Zdf) {       // G came from the tensor cores: the fallback needs the double-float Gram
        e = gram_df(Zdf, Zdf, d, m, G, part, st, nullptr, flag);
        if (e != cudaSuccess) return e;
    }
    const size_t smem_df = (size_t)3 * m * m * sizeof(float);
    e = allow_smem(cholesky_kernel<true>, smem_df);
    if (e != cudaSuccess) return e;
    note_launch();
    cholesky_kernel<true><<<1, kCholThreads, smem_df, st>>>(G, m, Rinv, flag, status);
    return cudaGetLastError();
}

cudaError_t apply_rinv(const float* V, const float* Rinv, int64_t d, int m, float* Q, cudaStream_t st) {
    if (V == Q || m > 128) return cudaErrorInvalidValue;
    const int threads = 2 * ((m + 31) / 32 * 32);
    const size_t smem = ((size_t)apply_xs_floats(m) + (size_t)m * kApplyRows) * sizeof(float);
    cudaError_t e = allow_smem(apply_rinv_kernel, smem);
    if (e != cudaSuccess) return e;
    note_launch();
    apply_rinv_kernel<<<ceil_div_i(d, kApplyRows), threads, smem, st>>>(V, Rinv, d, m, Q);
    return cudaGetLastError();
}

size_t jacobi_scratch_bytes(int m) {
    // evals (m f32) + Uf (m*m f32) + U64 (m*m f64) + lam (m f64) + sweeps, each 256-aligned
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    return al(m * 4) + al((size_t)m * m * 4) + al((size_t)m * m * 8) + al(m * 8) + al(4);
}

cudaError_t eigh_small(const double* G, int m, double* w, double* U, void* scratch, int* status, cudaStream_t st) {
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    char* p = static_cast<char*>(scratch);
    float* evals = reinterpret_cast<float*>(p);
    p += al(m * 4);
    float* Uf = reinterpret_cast<float*>(p);
    p += al((size_t)m * m * 4);
    double* U64 = reinterpret_cast<double*>(p);
    p += al((size_t)m * m * 8);
    double* lam = reinterpret_cast<double*>(p);
    p += al(m * 8);
    int* sweeps = reinterpret_cast<int*>(p);
    const int N = m + (m & 1);
    const size_t smem = (size_t)2 * N * (N + 1) * sizeof(float);
    cudaError_t e;
    if (N <= 32) {
        note_launch();
        jacobi_f32_kernel<32><<<1, 32, smem, st>>>(G, m, evals, Uf, sweeps, status);
    } else {
        e = allow_smem(jacobi_f32_kernel<512>, smem);
        if (e != cudaSuccess) return e;
        note_launch();
        jacobi_f32_kernel<512><<<1, 512, smem, st>>>(G, m, evals, Uf, sweeps, status);
    }
    note_launch();
    rayleigh_f64_kernel<<<m, 128, 0, st>>>(G, m, Uf, U64, lam);
    note_launch();
    sort_desc_kernel<<<1, 256, 0, st>>>(lam, U64, m, w, U);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Allocation-free eigensolve.  Some callers cannot allocate device memory at
// the point where they need the small eigensolve: code on a latency-critical
// path where a cudaMalloc (which may synchronise the device) is not
// acceptable, or hosts whose device memory is handed out by their own
// allocator.  For them the solve's
// scratch is one file-scope device array, sized for the largest m (128), that
// every device loading this library keeps until the process exits (each device
// has its own copy).  On one device the array is shared by all calls: calls
// that overlap on that GPU (e.g. enqueued on different streams) race on it and
// must be ordered by the caller.  Nothing in it needs to start at zero: every
// kernel of the solve writes its part of the scratch before reading it.
constexpr size_t kEighNoallocScratchBytes = 256 * 1024;
static __device__ __align__(256) unsigned char g_eigh_scratch[kEighNoallocScratchBytes];

size_t eigh_noalloc_scratch_bytes() { return kEighNoallocScratchBytes; }

cudaError_t eigh_small_noalloc(const double* G, int m, double* w, double* U, int* status, cudaStream_t st) {
    static_assert(kEighNoallocScratchBytes >= 1024 + 6 * 256 + (size_t)kMaxM * kMaxM * 12 + (size_t)kMaxM * 12,
                  "eigensolve scratch array too small for m = kMaxM");
    if (m < 1 || m > kMaxM || jacobi_scratch_bytes(m) > kEighNoallocScratchBytes) return cudaErrorInvalidValue;
    // Set-up, once per device and with that device current: host code may not
    // use g_eigh_scratch directly (its host-side name is only a stand-in), so
    // the device address is looked up and cached for the process (a
    // cudaDeviceReset after the first call is not supported: the cached
    // address would be stale).
    static std::mutex mu;
    static void* addr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_eigh_scratch);
            if (e != cudaSuccess) return e;
            addr[dev] = p;
        }
        scratch = addr[dev];
    }
    return eigh_small(G, m, w, U, scratch, status, st);
}

namespace {

// One step of the sequential power method, in one CTA (the method is meant for
// the small-scale protocol; every step reads one number back anyway).
constexpr int kSeqThreads = 1024;

__device__ double seq_block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kSeqThreads / 32; ++w) s += red[w];
        red[32] = s;
    }
    __syncthreads();
    const double s = red[32];
    __syncthreads();
    return s;
}

__global__ void __launch_bounds__(kSeqThreads) power_seq_kernel(float* __restrict__ V, int64_t d, int j,
                                                               float* __restrict__ y, double* __restrict__ diff) {
    __shared__ double red[33];
    __shared__ double cs[kMaxM];
    for (int pass = 0; pass < 2; ++pass) {             // classical Gram-Schmidt, twice
        for (int i = 0; i < j; ++i) {
            double p = 0.0;
            for (int64_t r = threadIdx.x; r < d; r += kSeqThreads) p += (double)V[(int64_t)i * d + r] * (double)y[r];
            const double c = seq_block_sum(p, red);
            if (threadIdx.x == 0) cs[i] = c;
        }
        __syncthreads();
        for (int64_t r = threadIdx.x; r < d; r += kSeqThreads) {
            double yr = (double)y[r];
            for (int i = 0; i < j; ++i) yr -= cs[i] * (double)V[(int64_t)i * d + r];
            y[r] = (float)yr;
        }
        __syncthreads();
    }
    double nn = 0.0;
    for (int64_t r = threadIdx.x; r < d; r += kSeqThreads) nn += (double)y[r] * (double)y[r];
    nn = seq_block_sum(nn, red);
    if (!(nn > 0.0)) {                                  // nothing left in the complement
        if (threadIdx.x == 0) *diff = 0.0;
        return;
    }
    const double inv = 1.0 / sqrt(nn);
    float* x = V + (int64_t)j * d;
    double dd = 0.0;
    for (int64_t r = threadIdx.x; r < d; r += kSeqThreads) {
        const double e = (double)y[r] * inv - (double)x[r];
        dd += e * e;
    }
    dd = seq_block_sum(dd, red);
    for (int64_t r = threadIdx.x; r < d; r += kSeqThreads) x[r] = (float)((double)y[r] * inv);
    if (threadIdx.x == 0) *diff = sqrt(dd);
}

}  // namespace

cudaError_t power_seq_update(float* V, int64_t d, int j, float* y, double* diff, cudaStream_t st) {
    if (j < 0 || j >= kMaxM) return cudaErrorInvalidValue;
    note_launch();
    power_seq_kernel<<<1, kSeqThreads, 0, st>>>(V, d, j, y, diff);
    return cudaGetLastError();
}

namespace {

// One CTA walks the blocks in chunks of its size; a block-wide exclusive scan
// of the keep flags gives each kept block its position, so the list comes out
// in ascending order.
constexpr int kSampleThreads = 1024;

__global__ void __launch_bounds__(kSampleThreads) sample_blocks_kernel(int64_t n, double fraction, uint64_t seed,
                                                                      int64_t forced, int* __restrict__ tile_rows) {
    __shared__ int warp_sum[kSampleThreads / 32];
    __shared__ int base;
    const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
    if (forced >= 0) {
        if (threadIdx.x == 0) tile_rows[0] = (int)(forced * 128);
        return;
    }
    const int64_t nt = (n + 127) / 128;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (int64_t c0 = 0; c0 < nt; c0 += kSampleThreads) {
        const int64_t t = c0 + threadIdx.x;
        const bool keep = t < nt && sample_block_kept(sample_block_u(seed, t), fraction);
        const unsigned ball = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) warp_sum[warp] = __popc(ball);
        __syncthreads();
        int before = 0;
        for (int w = 0; w < warp; ++w) before += warp_sum[w];
        const int pos = base + before + __popc(ball & ((1u << lane) - 1u));
        if (keep) tile_rows[pos] = (int)(t * 128);
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int w = 0; w < kSampleThreads / 32; ++w) tot += warp_sum[w];
            base += tot;
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t sample_blocks(int64_t n, double fraction, uint64_t seed, int64_t forced, int* tile_rows,
                          cudaStream_t st) {
    note_launch();
    sample_blocks_kernel<<<1, kSampleThreads, 0, st>>>(n, fraction, seed, forced, tile_rows);
    return cudaGetLastError();
}

cudaError_t rotate_and_sign(const float* Q, int64_t d, int m, const double* U, const double* w, int k, double inv_n,
                            float* E, double* lambda, cudaStream_t st) {
    note_launch();
    rotate_kernel<<<dim3(ceil_div_i(d, 256), k), 256, 0, st>>>(Q, d, m, U, k, E);
    note_launch();
    sign_kernel<<<k, 1024, 0, st>>>(E, d, w, inv_n, lambda);
    return cudaGetLastError();
}

cudaError_t oja_update(float* W, const float* Z, const double* S, int64_t d, int m, double c, cudaStream_t st,
                       const float* c_dev) {
    const size_t smem = ((size_t)m * m + (size_t)kOjaRows * (m + 1)) * sizeof(float);
    cudaError_t e = allow_smem(oja_update_kernel, smem);
    if (e != cudaSuccess) return e;
    note_launch();
    oja_update_kernel<<<ceil_div_i(d, kOjaRows), 256, smem, st>>>(W, Z, S, d, m, (float)c, c_dev);
    return cudaGetLastError();
}

cudaError_t primer_step_begin(PrimerStep* ps, int64_t per_epoch, int64_t b, double lr, double lr_offset,
                              cudaStream_t st) {
    note_launch();
    primer_step_kernel<<<1, 1, 0, st>>>(ps, per_epoch, b, lr, lr_offset);
    return cudaGetLastError();
}

cudaError_t primer_step_set(PrimerStep* ps, int64_t t, cudaStream_t st) {
    note_launch();
    primer_set_kernel<<<1, 1, 0, st>>>(ps, t);
    return cudaGetLastError();
}

cudaError_t eigengame_update(float* V, float* buf, const float* Z, const double* C, int64_t d, int m, double inv_b,
                             double lr, double mu, double* colnorm, cudaStream_t st) {
    // colnorm scratch layout: [coef m*m f32][alpha m f32][inv m float2][partials nblk*m float2]
    const int rows = eg_rows_per_block(d);
    const int nblk = ceil_div_i(d, rows);
    char* p = reinterpret_cast<char*>(colnorm);
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    float* coef = reinterpret_cast<float*>(p);
    p += al((size_t)m * m * 4);
    float* alpha = reinterpret_cast<float*>(p);
    p += al((size_t)m * 4);
    float2* inv = reinterpret_cast<float2*>(p);
    p += al((size_t)m * 8);
    float2* part = reinterpret_cast<float2*>(p);
    note_launch();
    eg_coef_kernel<<<m, kCoefThreads, 0, st>>>(C, m, inv_b, coef, alpha);
    const size_t smem = ((size_t)m * m + (size_t)m + 2 * (size_t)rows * (m + 1)) * 4;
    cudaError_t e = allow_smem(eg_step_kernel, smem);
    if (e != cudaSuccess) return e;
    note_launch();
    eg_step_kernel<<<nblk, 256, smem, st>>>(V, buf, Z, coef, alpha, d, m, rows, (float)inv_b, (float)lr,
                                                     (float)mu, part);
    note_launch();
    colnorm_reduce_kernel<<<m, kNormThreads, 0, st>>>(part, nblk, m, inv);
    note_launch();
    colscale_kernel<<<dim3(ceil_div_i(d, 256), m), 256, 0, st>>>(V, d, inv);
    return cudaGetLastError();
}

size_t eigengame_scratch_bytes(int64_t d, int m) {
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    return al((size_t)m * m * 4) + al((size_t)m * 4) + al((size_t)m * 8) +
           al((size_t)ceil_div_i(d, eg_rows_per_block(d)) * m * 8);
}

cudaError_t init_gaussian(float* V, int64_t d, int m, uint64_t seed, cudaStream_t st) {
    const int64_t count = d * m;
    const int64_t nthreads = (count + 3) / 4;
    note_launch();
    init_gaussian_kernel<<<ceil_div_i(nthreads, 256), 256, 0, st>>>(V, count, seed);
    return cudaGetLastError();
}

cudaError_t quantize_bf16(const float* X, int64_t n, int64_t d, int64_t ld_in, uint16_t* out, int64_t ld_out,
                          cudaStream_t st) {
    if (n == 0 || d == 0) return cudaSuccess;
    const bool vec = d % 8 == 0 && ld_in % 4 == 0 && ld_out % 8 == 0 && reinterpret_cast<uintptr_t>(X) % 16 == 0 &&
                     reinterpret_cast<uintptr_t>(out) % 16 == 0;
    if (vec) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int64_t groups = n * (d / 8);
        const int64_t blocks = std::min<int64_t>((groups + 255) / 256, (int64_t)sms * 8);
        note_launch();
        quantize_bf16_vec8_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, st>>>(X, n, d, ld_in, out,
                                                                                        ld_out);
        return cudaGetLastError();
    }
    const int gx = ceil_div_i(d, 256) > 64 ? 64 : ceil_div_i(d, 256);
    for (int64_t r0 = 0; r0 < n; r0 += 65535) {
        const int64_t rows = (n - r0) < 65535 ? (n - r0) : 65535;
        note_launch();
        quantize_bf16_kernel<<<dim3(gx, (unsigned)rows), 256, 0, st>>>(X + r0 * ld_in, rows, d, ld_in,
                                                                      out + r0 * ld_out, ld_out);
    }
    return cudaGetLastError();
}

cudaError_t quantize_fp8(const float* X, int64_t n, int64_t d, int64_t ld_in, uint8_t* out, int64_t ld_out,
                         float* scales, cudaStream_t st) {
    if (n == 0 || d == 0) return cudaSuccess;
    const bool vec = d % 4 == 0 && d <= 8 * 1024 && ld_in % 4 == 0 && ld_out % 4 == 0 &&
                     reinterpret_cast<uintptr_t>(X) % 16 == 0 && reinterpret_cast<uintptr_t>(out) % 4 == 0 &&
                     n <= 2147483647LL;
    if (vec) {
        const int vpt = (int)((d / 4 + 255) / 256);
        note_launch();
        switch (vpt) {
        case 1: quantize_fp8_vec4_kernel<1><<<(unsigned)n, 256, 0, st>>>(X, d, ld_in, out, ld_out, scales); break;
        case 2: quantize_fp8_vec4_kernel<2><<<(unsigned)n, 256, 0, st>>>(X, d, ld_in, out, ld_out, scales); break;
        case 3: quantize_fp8_vec4_kernel<3><<<(unsigned)n, 256, 0, st>>>(X, d, ld_in, out, ld_out, scales); break;
        case 4: quantize_fp8_vec4_kernel<4><<<(unsigned)n, 256, 0, st>>>(X, d, ld_in, out, ld_out, scales); break;
        case 5: quantize_fp8_vec4_kernel<5><<<(unsigned)n, 256, 0, st>>>(X, d, ld_in, out, ld_out, scales); break;
        case 6: quantize_fp8_vec4_kernel<6><<<(unsigned)n, 256, 0, st>>>(X, d, ld_in, out, ld_out, scales); break;
        case 7: quantize_fp8_vec4_kernel<7><<<(unsigned)n, 256, 0, st>>>(X, d, ld_in, out, ld_out, scales); break;
        default: quantize_fp8_vec4_kernel<8><<<(unsigned)n, 256, 0, st>>>(X, d, ld_in, out, ld_out, scales); break;
        }
        return cudaGetLastError();
    }
    for (int64_t r0 = 0; r0 < n; r0 += 2147483647LL) {
        const int64_t rows = n - r0;
        note_launch();
        quantize_fp8_kernel<<<(unsigned)rows, 256, 0, st>>>(X + r0 * ld_in, d, ld_in, out + r0 * ld_out, ld_out,
                                                            scales + r0);
    }
    return cudaGetLastError();
}

cudaError_t copy_f32(const float* src, float* dst, int64_t count, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    int blocks = ceil_div_i(count, 256);
    if (blocks > 4096) blocks = 4096;
    note_launch();
    copy_kernel<<<blocks, 256, 0, st>>>(src, dst, count);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ grouped launchers

cudaError_t grouped_gram(const GInst* gi, GTable gram_blocks, GTable reduce_blocks, int src, int max_m, bool gated,
                         cudaStream_t st) {
    (void)max_m;
    note_launch();
    gram_df_grouped_kernel<<<gram_blocks.total, 256, 0, st>>>(gi, gram_blocks, src, gated ? 1 : 0);
    note_launch();
    gram_reduce_grouped_kernel<<<reduce_blocks.total, 256, 0, st>>>(gi, reduce_blocks, gated ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t grouped_chol(const GInst* gi, int count, int max_m, bool near_identity, cudaStream_t st, bool span_only,
                         bool gated) {
    const size_t lda = (size_t)((max_m + 3) & ~3);
    size_t smem = ((size_t)2 * max_m * lda + (size_t)((max_m + kCB - 1) / kCB) * kCB * kCB + max_m) *
                  sizeof(float);
    if (!near_identity) smem = std::max(smem, (size_t)3 * max_m * max_m * sizeof(float));   // the fallback
    cudaError_t e = allow_smem(chol_blocked_grouped_kernel, smem);
    if (e != cudaSuccess) return e;
    note_launch();
    chol_blocked_grouped_kernel<<<count, kCBThreads, smem, st>>>(gi, near_identity ? 1 : 0, span_only ? 1 : 0,
                                                                  gated ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t grouped_apply_rinv(const GInst* gi, GTable blocks, int src, int dst, int max_m, cudaStream_t st,
                               bool split) {
    if (max_m > 128) return cudaErrorInvalidValue;
    const int threads = 2 * ((max_m + 31) / 32 * 32);
    const size_t smem = ((size_t)apply_xs_floats(max_m) + (size_t)max_m * kApplyRows) * sizeof(float);
    cudaError_t e = allow_smem(apply_rinv_grouped_kernel, smem);
    if (e != cudaSuccess) return e;
    note_launch();
    apply_rinv_grouped_kernel<<<blocks.total, threads, smem, st>>>(gi, blocks, src, dst, split ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t grouped_copy_v0(const GInst* gi, GTable dm_blocks, cudaStream_t st) {
    note_launch();
    copy_v0_grouped_kernel<<<dm_blocks.total, 256, 0, st>>>(gi, dm_blocks);
    return cudaGetLastError();
}

cudaError_t grouped_eigh(const GInst* gi, int count, GTable rayleigh_blocks, int max_m, cudaStream_t st) {
    const int N = max_m + (max_m & 1);
    const size_t smem = (size_t)2 * N * (N + 1) * sizeof(float);
    cudaError_t e = allow_smem(jacobi_grouped_kernel, smem);
    if (e != cudaSuccess) return e;
    note_launch();
    jacobi_grouped_kernel<<<count, 512, smem, st>>>(gi);
    note_launch();
    rayleigh_grouped_kernel<<<rayleigh_blocks.total, 128, 0, st>>>(gi, rayleigh_blocks);
    note_launch();
    sort_grouped_kernel<<<count, 256, 0, st>>>(gi);
    return cudaGetLastError();
}

cudaError_t grouped_rotate(const GInst* gi, GTable rotate_blocks, GTable sign_blocks, cudaStream_t st) {
    note_launch();
    rotate_grouped_kernel<<<rotate_blocks.total, 256, 0, st>>>(gi, rotate_blocks);
    note_launch();
    sign_grouped_kernel<<<sign_blocks.total, 1024, 0, st>>>(gi, sign_blocks);
    return cudaGetLastError();
}

cudaError_t grouped_copy_vout(const GInst* gi, GTable dm_blocks, cudaStream_t st) {
    note_launch();
    copy_vout_grouped_kernel<<<dm_blocks.total, 256, 0, st>>>(gi, dm_blocks);
    return cudaGetLastError();
}

// A grouped launch already spreads hundreds of instances over the GPU: row
// slices of 256 rows (not the single problem's 32, which fill the GPU with one
// narrow basis) keep the block count, and its scheduling cost, down.
constexpr int kGroupedGramRows = 256;

GShape grouped_shape(int64_t d, int m) {
    GShape s;
    s.gram_P = (int)std::min<int64_t>(gram_nslices(d, m), std::max<int64_t>(1, (d + kGroupedGramRows - 1) /
                                                                                  kGroupedGramRows));
    s.gram_T = (m + kGramTile - 1) / kGramTile;
    s.gram_L = gram_reduce_lanes(s.gram_P);
    s.gram_blocks = s.gram_T * s.gram_T * s.gram_P;
    s.reduce_blocks = ceil_div_i((int64_t)m * m * s.gram_L, 256);
    s.apply_blocks = ceil_div_i(d, kApplyRows);
    return s;
}

cudaError_t grouped_quantize_bf16(const float* const* X32, const int64_t* ld32, const GInst* gi, GTable blocks,
                                  cudaStream_t st) {
    note_launch();
    quantize_bf16_grouped_kernel<<<blocks.total, 256, 0, st>>>(X32, ld32, gi, blocks);
    return cudaGetLastError();
}

}  // namespace ppca
