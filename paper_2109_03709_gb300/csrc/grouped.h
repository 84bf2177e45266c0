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
    float* Zacc;              // [Sg][m_pad][Dt * 128] FP32 partials of Z, one per row group
    int Dt, Sg, kst, ntiles, nk;
    double* G;                // m x m
    float* Gf;                // m x m
    float* Rinv;              // m x m
    float* gram_part;         // gram_P x m x m x 2
    int gram_P, gram_T, gram_L;
    int* flag;                // CholeskyQR: the FP32 factor was rejected
    int* next;                // CholeskyQR: a second pass is needed (gated block power steps)
    int* status;              // device status word of the batch

    // the pPCA step (Algorithm 1, steps 2-5), Q = orth(V) held in Z
    int k;                    // components returned
    int xf32;                 // the step's data (XP) is FP32 (else BF16)
    const void* XP;           // the step's data: X as given, leading dimension ldp
    int64_t ldp;
    __nv_bfloat16* Q3;        // [3][m_pad][ldv]: Q as three BF16 pieces
    __nv_bfloat16* Y3;        // [3][m_pad][ldy]: Y = X Q as three BF16 pieces (transposed)
    float2* Gpart;            // [nparts][m_pad][m_pad]: double-float partials of Y^T Y
    int nparts;               // row chunks of Y^T Y (kGramChunk K-stages each)
    double* Gp;               // m x m: the projected Gram matrix
    float* evals;             // m: Jacobi eigenvalues (FP32)
    float* Uf;                // m x m: Jacobi eigenvectors (FP32)
    double* U64;              // m x m: FP64-polished eigenvectors
    double* lam;              // m: Rayleigh quotients
    int* sweeps;
    double* w;                // m: eigenvalues, descending
    double* U;                // m x m: eigenvectors, columns in the order of w
    float* E;                 // d x k output
    double* lambda;           // k output: w / n
    float* V_out;             // d x m output (NULL: none)
};

// K-stages (64 rows) of Y per partial of the grouped Y^T Y.
constexpr int kGramChunk = 64;

// TMA descriptors of one instance's X-pass (64-byte aligned in device memory).
struct alignas(64) GMaps {
    CUtensorMap xa;           // X, box 64 x 128 (Y = X V)
    CUtensorMap v;            // V pieces, box 64 x m_pad
    CUtensorMap xb;           // X, box 64 x 64 (Z = X^T Y)
    CUtensorMap y;            // Y^T, box 64 x m_pad
    CUtensorMap xp;           // the pPCA step's X: FP32 box 32 x 128, BF16 box 64 x 128
    CUtensorMap q3;           // Q pieces, box 64 x m_pad
    CUtensorMap y3;           // Y pieces, box 64 x m_pad
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
// gated: an instance's blocks do nothing while *next == 0 (its second pass is
// skipped).  grouped_chol: the first pass (near_identity false) redoes a
// rejected FP32 factor in double-float in the same block and sets *next when
// span_only; the second pass with gated writes R^-1 = I where *next == 0.
cudaError_t grouped_gram(const GInst* gi, GTable gram_blocks, GTable reduce_blocks, int src, int max_m,
                         bool gated, cudaStream_t st);
cudaError_t grouped_chol(const GInst* gi, int count, int max_m, bool near_identity, cudaStream_t st,
                         bool span_only = false, bool gated = false);
// split: also the BF16 rounding of the result into each instance's Vp.
cudaError_t grouped_apply_rinv(const GInst* gi, GTable blocks, int src, int dst, int max_m, cudaStream_t st,
                               bool split = false);
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

// ---- launchers (small.cu): the pPCA step's small kernels of every instance
cudaError_t grouped_eigh(const GInst* gi, int count, GTable rayleigh_blocks, int max_m, cudaStream_t st);
cudaError_t grouped_rotate(const GInst* gi, GTable rotate_blocks, GTable sign_blocks, cudaStream_t st);
cudaError_t grouped_copy_vout(const GInst* gi, GTable dm_blocks, cudaStream_t st);

// ---- launchers (pass_gram.cu): G = (X Q)^T (X Q) of every instance (split
// precision), over the instances with FP32 data (ygen32 items) and with BF16
// data (ygen16 items); gram items are (instance, chunk of kGramChunk K-stages)
cudaError_t grouped_projected_gram(const GInst* gi, const GMaps* maps, GTable ygen32, GTable ygen16, GTable gram_items,
                                   GTable reduce_blocks, int max_m, int* status, int num_sms, cudaStream_t st);
bool grouped_encode_gram_maps(const GInst& g, GMaps& out);

// ---- launchers (pass_tc.cu): the fast BF16 X-pass of every instance
// Q (held in Z) as three BF16 pieces Q3 (the pPCA step's split precision).
cudaError_t grouped_split_q(const GInst* gi, GTable blocks, cudaStream_t st);
cudaError_t grouped_xpass(const GInst* gi, const GMaps* maps, GTable xv_items, GTable xty_items,
                          GTable zred_blocks, int* status, int num_sms, cudaStream_t st);
bool grouped_encode_maps(const GInst& g, GMaps& out);

}  // namespace ppca
