// kernels.h -- internal launchers of the pPCA CUDA library.
//
// Every launcher enqueues on the given stream and returns the launch error.
// Matrices named V, Q, Z, W, E are d x m column-major FP32 (column j at
// offset j * d).  Small m x m matrices are row-major FP64 unless noted.
#pragma once

#include "common.cuh"

namespace ppca {

// ---- X-pass, SIMT reference kernels (pass_simt.cu) --------------------------
// Z = X[r0:r1]^T (X[r0:r1] V).  Ybuf: (r1 - r0) x m FP32 scratch.
// Zpart: nsplit * d * m * 2 floats of scratch.
struct SimtPassScratch {
    float* Y = nullptr;
    float* Zpart = nullptr;
    int nsplit = 1;             // split count the partial buffer was sized for
    int64_t zpart_floats = 0;   // capacity of Zpart
    int num_sms = 1;
};
size_t simt_pass_scratch_floats(int64_t rows, int64_t d, int m, int nsplit);
int simt_pass_nsplit(int64_t rows, int64_t d, int m, int num_sms);
cudaError_t xpass_simt(const XView& x, const float* V, int m, int64_t r0, int64_t r1, float* Z,
                       const SimtPassScratch& s, cudaStream_t st);

// ---- small dense kernels (small.cu) -------------------------------------------
// G = A^T B in double-float accumulation, A, B d x m column-major FP32,
// G m x m row-major FP64 (the rounded hi + lo pair) and, when Gf is given, its
// FP32 rounding.  part: scratch of gram_part_floats(d, m) floats (enough for
// every m' <= m as well).  run_if:
// device flag or NULL; when given, both kernels do nothing while *run_if == 0.
size_t gram_part_floats(int64_t d, int m);
cudaError_t gram_df(const float* A, const float* B, int64_t d, int m, double* G, float* part, cudaStream_t st,
                    float* Gf = nullptr, const int* run_if = nullptr);

// Cholesky G = R^T R (one CTA), writing X = R^-1 (upper, row-major FP32) to Rinv.
// FP32 blocked Cholesky of the diagonally scaled G (+ inverse), Rinv = R^-1.  With
// may_fall_back, a failed or ill-conditioned attempt sets *flag and the
// double-float Cholesky (launched right after, a no-op when *flag == 0) redoes it.
// Zdf: when G did not come from gram_df (tensor-core Gram), the d x m matrix
// whose double-float Gram the fallback recomputes into G first (gated by *flag,
// part as for gram_df); NULL otherwise.
// next (may be NULL, first pass): set to 0 when the accepted FP32 factor's
// conditioning bound is at most 2^10 (Q^T Q within ~1e-4 of I), else 1.
// run_if (may be NULL, second pass): while *run_if == 0 the factor is skipped
// and Rinv = I.
cudaError_t cholesky_adaptive(double* G, const float* Gf, int m, float* Rinv, bool may_fall_back, int* flag,
                              int* status, cudaStream_t st, const float* Zdf = nullptr, int64_t d = 0,
                              float* part = nullptr, int* next = nullptr, const int* run_if = nullptr);
// Q = V R^-1 as a product with the triangular inverse; Q must not alias V.
cudaError_t apply_rinv(const float* V, const float* Rinv, int64_t d, int m, float* Q, cudaStream_t st);

// Symmetric eigensolve (FP32 Jacobi + FP64 Rayleigh quotients), descending.
// G m x m FP64 row-major; w (m) FP64; U m x m column-major FP64.
// scratch: jacobi_scratch_bytes(m).
size_t jacobi_scratch_bytes(int m);
// Same solve with its scratch in a file-scope device array (no allocation);
// rejects m outside [1, kMaxM] with cudaErrorInvalidValue.
size_t eigh_noalloc_scratch_bytes();
cudaError_t eigh_small_noalloc(const double* G, int m, double* w, double* U, int* status, cudaStream_t st);
cudaError_t eigh_small(const double* G, int m, double* w, double* U, void* scratch, int* status,
                       cudaStream_t st);

// E[:, j] = Q U[:, j], j < k, signed by the largest-|entry| rule; lambda = w[:k] * inv_n.
cudaError_t rotate_and_sign(const float* Q, int64_t d, int m, const double* U, const double* w, int k,
                            double inv_n, float* E, double* lambda, cudaStream_t st);

// One step of the sequential power method for direction j of V (d x m
// column-major FP32): y <- y - V_<j (V_<j^T y) twice, x_new = y / |y|,
// *diff = |x_new - V[:, j]|, V[:, j] = x_new (FP64 arithmetic; y is modified).
// A zero y leaves V[:, j] and reports diff 0.
cudaError_t power_seq_update(float* V, int64_t d, int j, float* y, double* diff, cudaStream_t st);

// First rows of the kept 128-row blocks of an n-row matrix (ascending), by
// sample_block_kept; forced >= 0: keep that block alone (no block passed).
cudaError_t sample_blocks(int64_t n, double fraction, uint64_t seed, int64_t forced, int* tile_rows,
                          cudaStream_t st);

// Oja/Sanger update: W += c (Z - W triu(S)), S = W^T Z (m x m FP64 row-major), c = lr / b.
cudaError_t oja_update(float* W, const float* Z, const double* S, int64_t d, int m, double c,
                       cudaStream_t st, const float* c_dev = nullptr);

// Device state of graph-replayed minibatch steps (Oja, EigenGame): the step
// index, the first row of its minibatch, Oja's coefficient lr / (t + lr_offset) / b.
struct PrimerStep {
    int64_t t;
    int64_t row0;
    float c;
};
// One step's state from t (then t advances); setting t before a replay.
cudaError_t primer_step_begin(PrimerStep* ps, int64_t per_epoch, int64_t b, double lr, double lr_offset,
                              cudaStream_t st);
cudaError_t primer_step_set(PrimerStep* ps, int64_t t, cudaStream_t st);

// EigenGame update from Z = X_b^T X_b V and C = V^T Z (both unnormalised by b):
// MV = Z / b, Riemannian gradient, Nesterov momentum (buf), step lr, renormalise.
// colnorm: eigengame_scratch_bytes(d, m) bytes of scratch.
size_t eigengame_scratch_bytes(int64_t d, int m);
cudaError_t eigengame_update(float* V, float* buf, const float* Z, const double* C, int64_t d, int m,
                             double inv_b, double lr, double mu, double* colnorm, cudaStream_t st);

// Gaussian d x m basis from Philox4x32-10 (counter = element index, key = seed) + Box-Muller.
cudaError_t init_gaussian(float* V, int64_t d, int m, uint64_t seed, cudaStream_t st);

// Quantisers (data-format step).
cudaError_t quantize_bf16(const float* X, int64_t n, int64_t d, int64_t ld_in, uint16_t* out,
                          int64_t ld_out, cudaStream_t st);
cudaError_t quantize_fp8(const float* X, int64_t n, int64_t d, int64_t ld_in, uint8_t* out,
                         int64_t ld_out, float* scales, cudaStream_t st);

// Copy / zero helpers.
cudaError_t copy_f32(const float* src, float* dst, int64_t count, cudaStream_t st);

}  // namespace ppca
