// small.cu -- the small dense kernels of the pPCA path (d x m and m x m work).
//
//   gram_df          G = A^T B with double-float accumulation (CholeskyQR2's Gram,
//                    the projected Gram of the pPCA step, Oja's Y^T Y, EigenGame's C)
//   cholesky         G = R^T R in FP64 (one CTA)                 -- CholeskyQR2
//   apply_rinv       Q = V R^-1 by forward substitution          -- CholeskyQR2
//   eigh_small       parallel-order Jacobi (FP32 sweeps) + FP64 Rayleigh quotients
//                    -- the full-PCA of Algorithm 1, step 4
//   rotate_and_sign  E = Q U[:, :k], sign convention, lambda = w / n -- step 5
//   oja_update       generalised Oja (Sanger) rule, Section 2.2
//   eigengame_update EigenGame utility gradients (Section 2.3, Eq. 3), Riemannian
//                    projection, Nesterov momentum (Section 5), renormalisation
//   init_gaussian    Philox4x32-10 + Box-Muller starting basis
//   quantize_*       BF16 / FP8 E4M3 data formats
#include "kernels.h"

#include <cuda_fp8.h>
#include <math.h>

#include <mutex>

namespace ppca {

namespace {

constexpr int kGramTile = 32;        // output tile of gram_df
constexpr int kGramRows = 256;       // rows of A/B per slice

inline int gram_nslices(int64_t d) {
    int p = (int)((d + kGramRows - 1) / kGramRows);
    return p < 1 ? 1 : (p > 128 ? 128 : p);
}

// Exact product of two floats as an unevaluated sum p + e (FMA-based TwoProduct).
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

__global__ void gram_df_kernel(const float* __restrict__ A, const float* __restrict__ B, int64_t d, int m,
                               float* __restrict__ part, int64_t slice_rows) {
    __shared__ float As[32][kGramTile + 1];
    __shared__ float Bs[32][kGramTile + 1];
    const int ti = blockIdx.x, tj = blockIdx.y, p = blockIdx.z;
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
#pragma unroll 4
        for (int rr = 0; rr < 32; ++rr) {
#pragma unroll
            for (int a = 0; a < 2; ++a) {
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    float pp, pe;
                    two_prod(As[rr][ty * 2 + a], Bs[rr][tx * 2 + b], pp, pe);
                    df_add(hi[a][b], lo[a][b], pp);
                    lo[a][b] = __fadd_rn(lo[a][b], pe);
                }
            }
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

__global__ void gram_reduce_kernel(const float* __restrict__ part, int P, int m, bool sym, double* __restrict__ G) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m * m) return;
    const int i = idx / m, j = idx % m;
    const int src = (sym && i / kGramTile > j / kGramTile) ? j * m + i : idx;
    double s = 0.0;
    for (int p = 0; p < P; ++p) {
        const float* o = part + ((int64_t)p * m * m + src) * 2;
        s += (double)o[0] + (double)o[1];
    }
    G[idx] = s;
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
__global__ void __launch_bounds__(kCholThreads) cholesky_kernel(const double* __restrict__ G, int m,
                                                               float* __restrict__ Rinv, int* status) {
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

// Q = V X with X = R^-1 upper triangular (row-major): thread = one row of V,
// block column = 32 output columns; Q must not alias V.
constexpr int kApplyRows = 128;

__global__ void __launch_bounds__(kApplyRows) apply_rinv_kernel(const float* __restrict__ V,
                                                                 const float* __restrict__ Rinv, int64_t d, int m,
                                                                 float* __restrict__ Q) {
    extern __shared__ float xs[];   // (j0 + 32) x 32 slice of X
    const int j0 = blockIdx.y * 32;
    const int lmax = min(m, j0 + 32);
    for (int e = threadIdx.x; e < lmax * 32; e += blockDim.x) {
        const int l = e / 32, jj = e % 32;
        xs[e] = (j0 + jj < m) ? Rinv[l * m + j0 + jj] : 0.f;
    }
    __syncthreads();
    const int64_t r = (int64_t)blockIdx.x * kApplyRows + threadIdx.x;
    if (r >= d) return;
    float acc[32];
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) acc[jj] = 0.f;
    for (int l = 0; l < lmax; ++l) {
        const float v = V[(int64_t)l * d + r];
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) acc[jj] = __fmaf_rn(v, xs[l * 32 + jj], acc[jj]);
    }
#pragma unroll
    for (int jj = 0; jj < 32; ++jj)
        if (j0 + jj < m) Q[(int64_t)(j0 + jj) * d + r] = acc[jj];
}

// ------------------------------------------------------------------ Jacobi

// Parallel-order (round-robin) two-sided Jacobi in FP32 on N = m rounded up to
// even; the extra index is a decoupled zero row/column.  Each step applies N/2
// disjoint rotations J: A <- J^T A J is done block by block (every 2x2 block
// [rows p_t, q_t] x [cols p_u, q_u] needs only rotations t and u), so a step
// costs two barriers.  A rotation of pair (p, q) is skipped when
// |a_pq| <= tol * sqrt(|a_pp a_qq|), the relative criterion that keeps small
// eigenvalues accurate.  NT = 32 runs the whole solve in one warp.
constexpr int kJacobiMaxSweeps = 40;

__device__ __forceinline__ int rr_player(int pos, int step, int N) {
    return pos == 0 ? 0 : ((pos - 1 + step) % (N - 1)) + 1;
}

template <int NT>
__device__ __forceinline__ void jbar() {
    if (NT == 32) __syncwarp(); else __syncthreads();
}

template <int NT>
__global__ void __launch_bounds__(NT) jacobi_f32_kernel(const double* __restrict__ G, int m, float* __restrict__ evals,
                                                        float* __restrict__ Uf, int* sweeps_out, int* status) {
    extern __shared__ float js[];
    const int N = m + (m & 1);
    const int H = N / 2;
    const int S = N + 1;            // padded row stride: row and column sweeps are bank-conflict free
    float* A = js;                  // N x S
    float* U = A + N * S;           // N x S (column j = eigenvector j)
    float* cs = U + N * S;          // H cosines
    float* sn = cs + H;             // H sines
    float* dp = sn + H;             // H new a_pp
    float* dq = dp + H;             // H new a_qq
    int* pp = reinterpret_cast<int*>(dq + H);
    int* qq = pp + H;
    __shared__ int rotated;
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
            // rotations of the N/2 disjoint pairs of this step (classical angle)
            for (int t = threadIdx.x; t < H; t += NT) {
                int p = rr_player(t, step, N), q = rr_player(N - 1 - t, step, N);
                if (p > q) { const int x = p; p = q; q = x; }
                pp[t] = p;
                qq[t] = q;
                const float apq = A[p * S + q], app = A[p * S + p], aqq = A[q * S + q];
                float c = 1.f, s = 0.f, tt = 0.f;
                if (fabsf(apq) > 1e-30f && fabsf(apq) > tol * sqrtf(fabsf(app)) * sqrtf(fabsf(aqq))) {
                    const float tau = (aqq - app) / (2.0f * apq);
                    if (fabsf(tau) > 1e18f) {
                        tt = 0.5f / tau;
                    } else {
                        tt = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.0f + tau * tau));
                    }
                    c = 1.0f / sqrtf(1.0f + tt * tt);
                    s = tt * c;
                    rotated = 1;
                }
                cs[t] = c;
                sn[t] = s;
                dp[t] = app - tt * apq;
                dq[t] = aqq + tt * apq;
            }
            jbar<NT>();
            // rows p, q: A <- J^T A
            for (int t = threadIdx.x / 32; t < H; t += NT / 32) {      // one warp per pair
                const float s = sn[t];
                if (s == 0.f) continue;
                const float c = cs[t];
                const int p = pp[t], q = qq[t];
                for (int j = threadIdx.x % 32; j < N; j += 32) {
                    const float apj = A[p * S + j], aqj = A[q * S + j];
                    A[p * S + j] = c * apj - s * aqj;
                    A[q * S + j] = s * apj + c * aqj;
                }
            }
            jbar<NT>();
            // columns p, q: A <- A J, U <- U J; the pair's own 2x2 block gets the
            // exact zero and the tangent-formula diagonal
            for (int u = threadIdx.x / 32; u < H; u += NT / 32) {      // one warp per pair
                const float s = sn[u];
                if (s == 0.f) continue;
                const float c = cs[u];
                const int p = pp[u], q = qq[u];
                for (int i = threadIdx.x % 32; i < N; i += 32) {
                    if (i == p) {
                        A[p * S + p] = dp[u];
                        A[p * S + q] = 0.f;
                    } else if (i == q) {
                        A[q * S + p] = 0.f;
                        A[q * S + q] = dq[u];
                    } else {
                        const float aip = A[i * S + p], aiq = A[i * S + q];
                        A[i * S + p] = c * aip - s * aiq;
                        A[i * S + q] = s * aip + c * aiq;
                    }
                    const float uip = U[i * S + p], uiq = U[i * S + q];
                    U[i * S + p] = c * uip - s * uiq;
                    U[i * S + q] = s * uip + c * uiq;
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

// FP64 polish: u_j <- u_j / |u_j|, lambda_j = u_j^T G u_j (Rayleigh quotient).
__global__ void rayleigh_f64_kernel(const double* __restrict__ G, int m, const float* __restrict__ Uf,
                                    double* __restrict__ U64, double* __restrict__ lam) {
    __shared__ double u[kMaxM];
    __shared__ double red[32];
    const int j = blockIdx.x;
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

// Sort eigenpairs descending (stable in the index), in one CTA.
__global__ void sort_desc_kernel(const double* __restrict__ lam, const double* __restrict__ U64, int m,
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

// ------------------------------------------------------------------ rotate + sign

__global__ void rotate_kernel(const float* __restrict__ Q, int64_t d, int m, const double* __restrict__ U, int k,
                              float* __restrict__ E) {
    __shared__ float u[kMaxM];
    const int j = blockIdx.y;
    for (int i = threadIdx.x; i < m; i += blockDim.x) u[i] = (float)U[j * m + i];
    __syncthreads();
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= d) return;
    float s = 0.f;
    for (int i = 0; i < m; ++i) s = __fmaf_rn(Q[(int64_t)i * d + r], u[i], s);
    E[(int64_t)j * d + r] = s;
}

__global__ void sign_kernel(float* __restrict__ E, int64_t d, const double* __restrict__ w, double inv_n,
                            double* __restrict__ lambda) {
    const int j = blockIdx.x;
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

// ------------------------------------------------------------------ Oja / Sanger

constexpr int kRowThreads = 64;

__global__ void oja_update_kernel(float* __restrict__ W, const float* __restrict__ Z, const double* __restrict__ S,
                                  int64_t d, int m, float c) {
    extern __shared__ float sm[];
    float* Ss = sm;                        // m x m (row-major)
    float* w = sm + m * m;                 // m x kRowThreads
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) Ss[e] = (float)S[e];
    __syncthreads();
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= d) return;
    const int t = threadIdx.x;
    for (int j = 0; j < m; ++j) w[j * kRowThreads + t] = W[(int64_t)j * d + r];
    for (int j = 0; j < m; ++j) {
        float acc = 0.f;
        for (int l = 0; l <= j; ++l) acc = __fmaf_rn(w[l * kRowThreads + t], Ss[l * m + j], acc);
        const float z = Z[(int64_t)j * d + r];
        W[(int64_t)j * d + r] = w[j * kRowThreads + t] + c * (z - acc);
    }
}

// ------------------------------------------------------------------ EigenGame

// coef[i][j] = C_ij / C_ii (i < j), alpha_j = 2 C_jj - 2 sum_{i<j} C_ij^2 / C_ii, C scaled by 1/b.
__global__ void eg_coef_kernel(const double* __restrict__ C, int m, double inv_b, float* __restrict__ coef,
                               float* __restrict__ alpha) {
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int i = e / m, j = e % m;
        const double cii = C[i * m + i] * inv_b;
        const double cij = 0.5 * (C[i * m + j] + C[j * m + i]) * inv_b;
        coef[e] = (i < j && cii != 0.0) ? (float)(cij / cii) : 0.f;
    }
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        double a = 2.0 * C[j * m + j] * inv_b;
        for (int i = 0; i < j; ++i) {
            const double cii = C[i * m + i] * inv_b;
            const double cij = 0.5 * (C[i * m + j] + C[j * m + i]) * inv_b;
            if (cii != 0.0) a -= 2.0 * cij * cij / cii;
        }
        alpha[j] = (float)a;
    }
}

__global__ void eg_step_kernel(float* __restrict__ V, float* __restrict__ buf, const float* __restrict__ Z,
                               const float* __restrict__ coef_g, const float* __restrict__ alpha_g, int64_t d, int m,
                               float inv_b, float lr, float mu, double* __restrict__ colpart) {
    extern __shared__ float sm[];
    float* coef = sm;                      // m x m
    float* alpha = coef + m * m;           // m
    float* mv = alpha + m;                 // m x kRowThreads
    __shared__ double red[kMaxM];
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) coef[e] = coef_g[e];
    for (int e = threadIdx.x; e < m; e += blockDim.x) { alpha[e] = alpha_g[e]; red[e] = 0.0; }
    __syncthreads();
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int t = threadIdx.x;
    const bool live = r < d;
    if (live)
        for (int j = 0; j < m; ++j) mv[j * kRowThreads + t] = Z[(int64_t)j * d + r] * inv_b;
    for (int j = 0; j < m; ++j) {
        float vn = 0.f;
        if (live) {
            float g = 2.f * mv[j * kRowThreads + t];
            for (int i = 0; i < j; ++i) g = __fmaf_rn(-2.f * coef[i * m + j], mv[i * kRowThreads + t], g);
            const float v = V[(int64_t)j * d + r];
            g = __fmaf_rn(-alpha[j], v, g);                       // Riemannian projection
            const float b = __fmaf_rn(mu, buf[(int64_t)j * d + r], g);
            buf[(int64_t)j * d + r] = b;
            vn = __fmaf_rn(lr, __fmaf_rn(mu, b, g), v);           // Nesterov step
            V[(int64_t)j * d + r] = vn;
        }
        // column norm^2 partial of this block
        double x = (double)vn * (double)vn;
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffff, x, o);
        if ((t & 31) == 0) atomicAdd(&red[j], x);   // within the block only: fixed set of warps
    }
    __syncthreads();
    for (int j = threadIdx.x; j < m; j += blockDim.x) colpart[(int64_t)blockIdx.x * m + j] = red[j];
}

__global__ void colnorm_reduce_kernel(const double* __restrict__ colpart, int nblk, int m, double* __restrict__ nrm) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += colpart[(int64_t)b * m + j];
    nrm[j] = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
}

__global__ void colscale_kernel(float* __restrict__ V, int64_t d, int m, const double* __restrict__ inv) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= d) return;
    for (int j = 0; j < m; ++j) V[(int64_t)j * d + r] = (float)((double)V[(int64_t)j * d + r] * inv[j]);
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

__global__ void copy_kernel(const float* __restrict__ s, float* __restrict__ d, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d[i] = s[i];
}

template <typename K>
cudaError_t allow_smem(K kernel, size_t bytes) {
    if (bytes <= 32 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

// ============================================================================ launchers

size_t gram_part_floats(int64_t d, int m) { return (size_t)gram_nslices(d) * m * m * 2; }

cudaError_t gram_df(const float* A, const float* B, int64_t d, int m, double* G, float* part, cudaStream_t st) {
    const int P = gram_nslices(d);
    const int64_t slice = (d + P - 1) / P;
    const int T = (m + kGramTile - 1) / kGramTile;
    note_launch();
    gram_df_kernel<<<dim3(T, T, P), 256, 0, st>>>(A, B, d, m, part, slice);
    note_launch();
    gram_reduce_kernel<<<(m * m + 255) / 256, 256, 0, st>>>(part, P, m, A == B, G);
    return cudaGetLastError();
}

cudaError_t cholesky(const double* G, int m, float* Rinv, bool double_float, int* status, cudaStream_t st) {
    cudaError_t e;
    if (double_float) {
        const size_t smem = (size_t)3 * m * m * sizeof(float);
        e = allow_smem(cholesky_kernel<true>, smem);
        if (e != cudaSuccess) return e;
        note_launch();
        cholesky_kernel<true><<<1, kCholThreads, smem, st>>>(G, m, Rinv, status);
    } else {
        const size_t smem = (size_t)2 * m * m * sizeof(float);
        e = allow_smem(cholesky_kernel<false>, smem);
        if (e != cudaSuccess) return e;
        note_launch();
        cholesky_kernel<false><<<1, kCholThreads, smem, st>>>(G, m, Rinv, status);
    }
    return cudaGetLastError();
}

cudaError_t apply_rinv(const float* V, const float* Rinv, int64_t d, int m, float* Q, cudaStream_t st) {
    if (V == Q) return cudaErrorInvalidValue;
    const size_t smem = (size_t)m * 32 * sizeof(float);
    note_launch();
    apply_rinv_kernel<<<dim3(ceil_div_i(d, kApplyRows), ceil_div_i(m, 32)), kApplyRows, smem, st>>>(V, Rinv, d, m,
                                                                                                     Q);
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
    const size_t smem = (size_t)2 * N * (N + 1) * sizeof(float) + (size_t)(N / 2) * (4 * sizeof(float) + 2 * sizeof(int));
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
// the point where they need the small eigensolve: code running while a stream
// is being captured into a CUDA graph, code on a latency-critical path where a
// cudaMalloc (which may synchronise the device) is not acceptable, or hosts
// whose memory is handed out by their own allocator.  For them the solve's
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
    // the device address is looked up and cached.
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

cudaError_t rotate_and_sign(const float* Q, int64_t d, int m, const double* U, const double* w, int k, double inv_n,
                            float* E, double* lambda, cudaStream_t st) {
    note_launch();
    rotate_kernel<<<dim3(ceil_div_i(d, 256), k), 256, 0, st>>>(Q, d, m, U, k, E);
    note_launch();
    sign_kernel<<<k, 1024, 0, st>>>(E, d, w, inv_n, lambda);
    return cudaGetLastError();
}

cudaError_t oja_update(float* W, const float* Z, const double* S, int64_t d, int m, double c, cudaStream_t st) {
    const size_t smem = (size_t)m * m * sizeof(float) + (size_t)m * kRowThreads * sizeof(float);
    cudaError_t e = allow_smem(oja_update_kernel, smem);
    if (e != cudaSuccess) return e;
    note_launch();
    oja_update_kernel<<<ceil_div_i(d, kRowThreads), kRowThreads, smem, st>>>(W, Z, S, d, m, (float)c);
    return cudaGetLastError();
}

cudaError_t eigengame_update(float* V, float* buf, const float* Z, const double* C, int64_t d, int m, double inv_b,
                             double lr, double mu, double* colnorm, cudaStream_t st) {
    // colnorm scratch layout: [coef m*m f32][alpha m f32][inv m f64][partials nblk*m f64]
    const int nblk = ceil_div_i(d, kRowThreads);
    char* p = reinterpret_cast<char*>(colnorm);
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    float* coef = reinterpret_cast<float*>(p);
    p += al((size_t)m * m * 4);
    float* alpha = reinterpret_cast<float*>(p);
    p += al((size_t)m * 4);
    double* inv = reinterpret_cast<double*>(p);
    p += al((size_t)m * 8);
    double* part = reinterpret_cast<double*>(p);
    note_launch();
    eg_coef_kernel<<<1, 256, 0, st>>>(C, m, inv_b, coef, alpha);
    const size_t smem = (size_t)m * m * 4 + (size_t)m * 4 + (size_t)m * kRowThreads * 4;
    cudaError_t e = allow_smem(eg_step_kernel, smem);
    if (e != cudaSuccess) return e;
    note_launch();
    eg_step_kernel<<<nblk, kRowThreads, smem, st>>>(V, buf, Z, coef, alpha, d, m, (float)inv_b, (float)lr,
                                                     (float)mu, part);
    note_launch();
    colnorm_reduce_kernel<<<1, 128, 0, st>>>(part, nblk, m, inv);
    note_launch();
    colscale_kernel<<<ceil_div_i(d, 256), 256, 0, st>>>(V, d, m, inv);
    return cudaGetLastError();
}

size_t eigengame_scratch_bytes(int64_t d, int m) {
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    return al((size_t)m * m * 4) + al((size_t)m * 4) + al((size_t)m * 8) +
           al((size_t)ceil_div_i(d, kRowThreads) * m * 8);
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

}  // namespace ppca
