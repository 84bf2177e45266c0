// pass_tc.h -- tensor-core (tcgen05 + TMA) X-passes and projected Gram (internal).
#pragma once

#include "common.cuh"

namespace ppca {

struct TcPassScratch {
    void* vp = nullptr;     // V pieces, [3][128][round_up(d, 8)] BF16
    void* yt = nullptr;     // Y^T pieces, [3][128][round_up(n, 128)] BF16
    void* zacc = nullptr;   // double-float Z partials, [row group][d slice * 128][128] x 2 FP32
                            // (also split-K partials of Y and the projected Gram's partials)
    size_t z_bytes = 0;     // capacity of zacc
    int* flags = nullptr;   // fused pass: ready[tiles], consumed[tiles]
};

// Schedule of the fast (one-piece) pass; zero fields mean "library choice".
struct TcSchedule {
    int fused = -1;         // 1: fused single-read kernel, 0: two GEMM kernels, -1: choose
    int producers = 0;      // CTAs running the Y = X V pipeline in the fused kernel
    int window = 0;         // tiles a producer may run ahead of the slowest consumer
    int flush = 0;          // projected Gram and fused pass: K-stages per accumulator fold (0: default)
    int engine = 0;         // 0: library choice, 1: tensor cores, 2: CUDA cores
    int kparts = 0;         // fused kernel: K parts per producer tile (2: two K halves; else 1)
    int l2_keep = 0;        // fused kernel: percent of a tile's K-stages loaded evict_last (0: from the L2 size)
    int fp8_mma = -1;       // FP8 data, FAST: 1 / -1 the FP8 tensor cores (kind::f8f6f4), 0 widening to BF16
};

size_t tc_pass_scratch_bytes(int64_t n, int64_t d, int m, int num_sms);
TcPassScratch tc_pass_scratch_carve(void* base, int64_t n, int64_t d, int m, int num_sms);
bool tc_pass_supported(const XView& x, int m);
// G = (X[r0:r1] Q)^T (X[r0:r1] Q), m x m FP64 row-major (symmetric), for BF16 or
// FP32 X.  ACCURATE/AUTO: split-precision products (about 2^-24); FAST: one BF16
// piece of Q (BF16 X) or two pieces of each operand (FP32 X).  flush <= 0: the
// library's choice of K-stages per accumulator flush.
cudaError_t projected_gram_tc(const XView& x, const float* Q, int m, int64_t r0, int64_t r1, double* G,
                              ppca_precision prec, int flush, const TcPassScratch& s, int* status, int num_sms,
                              cudaStream_t st);
// G = Z^T Z (m x m FP64, and its FP32 rounding in Gf) for Z d x m column-major
// FP32 on the tensor cores: three BF16 pieces of Z, six piece products, about
// 2^-24 relative to |z_i| |z_j|.  Uses s.vp and s.zacc.
cudaError_t gram_tc(const float* Z, int64_t d, int m, double* G, float* Gf, const TcPassScratch& s, int* status,
                    int num_sms, cudaStream_t st);
// The same over the nsel 128-row blocks of X whose first rows are listed in
// tile_row (device array, rows < n; a block past row n - 1 reads zeros).
cudaError_t projected_gram_tc_blocks(const XView& x, const float* Q, int m, const int* tile_row, int nsel, double* G,
                                     ppca_precision prec, int flush, const TcPassScratch& s, int* status,
                                     int num_sms, cudaStream_t st);
// Limit of the bounded device waits of the tensor-core kernels on the current
// device (ns = 0: the default 2 s), one setter per translation unit.
cudaError_t pass_tc_set_wait_limit(uint64_t ns);
cudaError_t pass_gram_set_wait_limit(uint64_t ns);
// row0_dev (device, may be NULL): the kernels read the first row of the rows
// [r0, r1) there instead of taking r0 (r1 - r0 a multiple of 128; FP32 or
// BF16 data; the two-kernel forms), so a captured pass can serve any batch.
cudaError_t xpass_tc(const XView& x, const float* V, int m, int64_t r0, int64_t r1, float* Z, ppca_precision prec,
                     const TcPassScratch& s, const TcSchedule& sched, int* status, int num_sms, cudaStream_t st,
                     const int64_t* row0_dev = nullptr);
// True when the device-first-row form of a pass over `rows` rows runs the same
// kernels (and so gives the same bits) as the ordinary form.
bool xpass_tc_row0_same(const XView& x, int64_t rows, ppca_precision prec, const TcSchedule& sched, int num_sms);

}  // namespace ppca
