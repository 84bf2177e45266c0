// pass_simt.cu -- CUDA-core X-pass: Z = X[r0:r1]^T (X[r0:r1] V), FP32 FMA.
//
// The product X^T X V is the inner step of every primer (Section 2.1: M x with
// M = X^T X; Section 2.2: x x^T w summed over the batch; Section 2.3: M v_j).
// This version is the exact-FP32 path: it reads X twice (once for Y = X V,
// once for Z = X^T Y) and keeps Y in global memory.  The tensor-core pass in
// pass_tc.cu reads X once; this one covers shapes it does not take and serves
// as the FP32 reference on the device.
//
// Accuracy: each thread accumulates at most kFlushRows products in FP32 and
// then folds the block sum into a double-float (hi, lo) pair; the split-K
// partials are reduced in double-float too, so the result is within a few FP32
// ulps of the exact sum of the rounded FP32 products.
#include "kernels.h"

namespace ppca {

namespace {

constexpr int BM = 64, BN = 64, BK = 16;
constexpr int kFlushRows = 256;

// Y (rows x m, row-major, stride m) = X[r0:r0+rows] V
__global__ void __launch_bounds__(256) xv_kernel(XView x, const float* __restrict__ V, int m, int64_t r0,
                                                 int64_t rows, float* __restrict__ Y) {
    __shared__ float Xs[BK][BM + 4];
    __shared__ float Vs[BK][BN + 4];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int64_t rb = (int64_t)blockIdx.x * BM;
    const int cb = blockIdx.y * BN;
    float acc[4][4] = {};
    for (int64_t k0 = 0; k0 < x.d; k0 += BK) {
        for (int e = threadIdx.x; e < BM * BK; e += 256) {
            const int kk = e % BK, rr = e / BK;
            const int64_t r = rb + rr, j = k0 + kk;
            Xs[kk][rr] = (r < rows && j < x.d) ? load_x(x, r0 + r, j) : 0.f;
        }
        for (int e = threadIdx.x; e < BN * BK; e += 256) {
            const int kk = e % BK, cc = e / BK;
            const int64_t j = k0 + kk;
            const int c = cb + cc;
            Vs[kk][cc] = (c < m && j < x.d) ? V[(int64_t)c * x.d + j] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = Xs[kk][ty * 4 + i];
#pragma unroll
            for (int i = 0; i < 4; ++i) b[i] = Vs[kk][tx * 4 + i];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = __fmaf_rn(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t r = rb + ty * 4 + i;
        if (r >= rows) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = cb + tx * 4 + j;
            if (c < m) Y[r * m + c] = acc[i][j];
        }
    }
}

// Partial of Z[j][c] = sum_r X[r][j] Y[r][c] over the rows of split s.
__global__ void __launch_bounds__(256) xty_kernel(XView x, const float* __restrict__ Y, int m, int64_t r0,
                                                  int64_t rows, int64_t split_rows, float* __restrict__ part) {
    __shared__ float Xs[BK][BM + 4];
    __shared__ float Ys[BK][BN + 4];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int64_t jb = (int64_t)blockIdx.x * BM;
    const int cb = blockIdx.y * BN;
    const int s = blockIdx.z;
    const int64_t rbeg = (int64_t)s * split_rows;
    const int64_t rend = min(rows, rbeg + split_rows);
    float acc[4][4] = {}, hi[4][4] = {}, lo[4][4] = {};
    int since = 0;
    for (int64_t k0 = rbeg; k0 < rend; k0 += BK) {
        for (int e = threadIdx.x; e < BM * BK; e += 256) {
            const int jj = e % BM, kk = e / BM;
            const int64_t r = k0 + kk, j = jb + jj;
            Xs[kk][jj] = (r < rend && j < x.d) ? load_x(x, r0 + r, j) : 0.f;
        }
        for (int e = threadIdx.x; e < BN * BK; e += 256) {
            const int cc = e % BN, kk = e / BN;
            const int64_t r = k0 + kk;
            const int c = cb + cc;
            Ys[kk][cc] = (r < rend && c < m) ? Y[r * m + c] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = Xs[kk][ty * 4 + i];
#pragma unroll
            for (int i = 0; i < 4; ++i) b[i] = Ys[kk][tx * 4 + i];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = __fmaf_rn(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
        since += BK;
        if (since >= kFlushRows) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    df_add(hi[i][j], lo[i][j], acc[i][j]);
                    acc[i][j] = 0.f;
                }
            since = 0;
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) df_add(hi[i][j], lo[i][j], acc[i][j]);
    // part layout: [s][c][j] pairs (hi, lo), Z column-major per split
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t j = jb + ty * 4 + i;
        if (j >= x.d) continue;
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int c = cb + tx * 4 + jj;
            if (c >= m) continue;
            float* o = part + (((int64_t)s * m + c) * x.d + j) * 2;
            o[0] = hi[i][jj];
            o[1] = lo[i][jj];
        }
    }
}

__global__ void split_reduce_kernel(const float* __restrict__ part, int nsplit, int64_t count, float* __restrict__ Z) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        float hi = 0.f, lo = 0.f;
        for (int s = 0; s < nsplit; ++s) {
            const float* o = part + ((int64_t)s * count + i) * 2;
            df_add(hi, lo, o[0]);
            df_add(hi, lo, o[1]);
        }
        Z[i] = __fadd_rn(hi, lo);
    }
}

}  // namespace

int simt_pass_nsplit(int64_t rows, int64_t d, int m, int num_sms) {
    const int64_t tiles = (int64_t)ceil_div_i(d, BM) * ceil_div_i(m, BN);
    int64_t want = (4LL * num_sms + tiles - 1) / tiles;           // about 4 waves
    const int64_t by_rows = (rows + kFlushRows - 1) / kFlushRows;
    if (want > by_rows) want = by_rows;
    // keep the partials under 256 MB
    const int64_t cap = (256LL << 20) / ((int64_t)d * m * 8 + 1);
    if (want > cap) want = cap;
    return want < 1 ? 1 : (int)want;
}

size_t simt_pass_scratch_floats(int64_t rows, int64_t d, int m, int nsplit) {
    return (size_t)rows * m + (size_t)nsplit * d * m * 2;
}

cudaError_t xpass_simt(const XView& x, const float* V, int m, int64_t r0, int64_t r1, float* Z,
                       const SimtPassScratch& s, cudaStream_t st) {
    const int64_t rows = r1 - r0;
    if (rows <= 0) return cudaErrorInvalidValue;
    for (int64_t rb = 0; rb < rows; rb += 65535LL * BM) {
        const int64_t chunk = (rows - rb) < 65535LL * BM ? (rows - rb) : 65535LL * BM;
        note_launch();
        xv_kernel<<<dim3(ceil_div_i(chunk, BM), ceil_div_i(m, BN)), 256, 0, st>>>(x, V, m, r0 + rb, chunk,
                                                                                   s.Y + rb * m);
    }
    // The split depends only on this problem's shape (not on how large the
    // workspace is), so a problem gives the same bits alone or in a batch.
    int want = simt_pass_nsplit(x.n, x.d, m, s.num_sms);
    while (want > 1 && (int64_t)want * x.d * m * 2 > s.zpart_floats) --want;
    const int64_t split_rows = ((rows + want - 1) / want + BK - 1) / BK * BK;
    const int nsplit = (int)((rows + split_rows - 1) / split_rows);
    note_launch();
    xty_kernel<<<dim3(ceil_div_i(x.d, BM), ceil_div_i(m, BN), nsplit), 256, 0, st>>>(x, s.Y, m, r0, rows, split_rows,
                                                                                     s.Zpart);
    const int64_t count = x.d * m;
    int blocks = ceil_div_i(count, 256);
    if (blocks > 2048) blocks = 2048;
    note_launch();
    split_reduce_kernel<<<blocks, 256, 0, st>>>(s.Zpart, nsplit, count, Z);
    return cudaGetLastError();
}

}  // namespace ppca
