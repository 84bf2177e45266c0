// grouped.h -- grouped launches: one kernel launch works on many independent
// problems ("instances") of uneven size (internal).
//
// Each instance is described by a GInst in device memory.  A grouped launch of
// some kernel kind gives instance i the blocks [base[i], base[i + 1]) of its
// grid (base a prefix table on the device, count + 1 entries): block b belongs
// to the instance found by binary search and is that instance's block
// b - base[i], which the kernel body handles exactly as the single-instance
// launch would.  Persistent kernels (the X-pass) use the same tables over work
// items instead of blocks.
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace ppca {

struct GInst {
    const void* X;            // priming data: BF16, n x d row-major, leading dimension ld
    int64_t n, d, ld;
    int m, m_pad;
    const float* V0;          // d x m starting basis (NULL: drawn from the instance's seed)
    float* V;                 // d x m column-major: the primed basis
    float* Z;                 // d x m: the pass output
    float* T;                 // d x m: CholeskyQR's first factor
    __nv_bfloat16* Vp;        // [m_pad][ldv]: V rounded to BF16
    int64_t ldv;
    __nv_bfloat16* Yt;        // [m_pad][ldy]: Y^T rounded to BF16
    int64_t ldy;
    float* Zacc;              // [Sg][m_pad][Dt * 128] double-float partials of Z
    int Dt, Sg, kst, ntiles, nk;
    double* G;                // m x m
    float* Gf;                // m x m
    float* Rinv;              // m x m
    float* gram_part;         // gram_P x m x m x 2
    int gram_P, gram_T, gram_L;
    int* flag;                // CholeskyQR: the FP32 factor was rejected
    int* status;              // device status word of the batch
};

// TMA descriptors of one instance's X-pass (64-byte aligned in device memory).
struct alignas(64) GMaps {
    CUtensorMap xa;           // X, box 64 x 128 (Y = X V)
    CUtensorMap v;            // V pieces, box 64 x m_pad
    CUtensorMap xb;           // X, box 64 x 64 (Z = X^T Y)
    CUtensorMap y;            // Y^T, box 64 x m_pad
};

// A grouped launch's block (or work item) table.
struct GTable {
    const int* base;          // count + 1 entries, base[count] = total
    int count;
    int total;
};

__device__ __forceinline__ int group_find(const GTable& t, int b) {
    int lo = 0, hi = t.count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (t.base[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Which d x m array of an instance a grouped CholeskyQR round reads or writes.
enum GArray : int { kGV = 0, kGZ = 1, kGT = 2 };

__host__ __device__ inline float* garray(const GInst& g, int which) {
    return which == kGV ? g.V : (which == kGZ ? g.Z : g.T);
}

// ---- launchers (small.cu): CholeskyQR2 of every instance, src -> dst (V, Z or T)
cudaError_t grouped_gram(const GInst* gi, GTable gram_blocks, GTable reduce_blocks, int src, int max_m,
                         bool gated, cudaStream_t st);
cudaError_t grouped_chol(const GInst* gi, int count, int max_m, bool near_identity, cudaStream_t st);
cudaError_t grouped_chol_fallback(const GInst* gi, int count, int max_m, cudaStream_t st);
cudaError_t grouped_apply_rinv(const GInst* gi, GTable blocks, int src, int dst, int max_m, cudaStream_t st);
cudaError_t grouped_quantize_bf16(const float* const* X32, const int64_t* ld32, const GInst* gi, GTable blocks,
                                  cudaStream_t st);
cudaError_t grouped_copy_v0(const GInst* gi, GTable dm_blocks, cudaStream_t st);

// Per-instance launch shapes of the grouped CholeskyQR kernels: row slices P,
// output tiles T (per side) and reduce lanes L of the Gram; blocks of the Gram,
// of its reduction and of Q = V R^-1.
struct GShape {
    int gram_P, gram_T, gram_L, gram_blocks, reduce_blocks, apply_blocks;
};
GShape grouped_shape(int64_t d, int m);

// ---- launchers (pass_tc.cu): the fast BF16 X-pass of every instance
cudaError_t grouped_split_v(const GInst* gi, GTable blocks, cudaStream_t st);
cudaError_t grouped_xpass(const GInst* gi, const GMaps* maps, GTable xv_items, GTable xty_items,
                          GTable zred_blocks, int* status, int num_sms, cudaStream_t st);
bool grouped_encode_maps(const GInst& g, GMaps& out);

}  // namespace ppca
