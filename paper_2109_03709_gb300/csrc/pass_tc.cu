// pass_tc.cu -- tensor-core X-pass Z = X^T (X V) on tcgen05 + TMA: BF16 data
// (the two kernels below, and the fused single-read pass further down), FP8
// E4M3 data (widened to BF16 in shared memory) and FP32 data (3xTF32).
//
// The product X^T X V (Section 2.1's M x with M = X^T X; the minibatch sums
// of Sections 2.2-2.3; the projection of Algorithm 1, step 3) is computed as
//
//   xv_tc   Y = X V     persistent over 128-row tiles of X; A = X tile
//                       (K-major, TMA, 128B swizzle), B = V pieces (K-major),
//                       FP32 accumulator in TMEM (double-buffered), epilogue
//                       splits Y into S BF16 pieces written column-major (Y^T).
//   xty_tc  Z = X^T Y   one CTA per (128-column slice of d, row group); A = the
//                       same X tiles read MN-major, B = Y^T pieces; the FP32
//                       accumulator lives in TMEM for a block of rows and is then
//                       folded into a double-float partial in global memory.
//   reduce  Z = sum over row groups of the double-float partials.
//
// Split precision: with S = 3, V (and Y) are split into hi + mid + lo BF16
// pieces (24 significand bits); X is exact in BF16, so the products carry
// FP32-level accuracy ("BF16x3").  S = 1 is the fast priming pass.
//
// Warp roles (192 threads): warp 0 issues TMA, warp 1 owns TMEM and issues the
// MMAs (one thread), warps 2-5 are the epilogue (TMEM lane quarter = warp % 4).
// Every wait is bounded by a 2 s clock; on timeout the kernel records
// kDevWaitTimeout, drains its copies, frees TMEM and returns.
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "grouped.h"
#include "pass_tc.h"
#include "tc_host.h"
#include "tc_ptx.cuh"

namespace ppca {

namespace {

constexpr int kThreads = 192;
constexpr int kThreadsFp8 = 448;          // + eight transform warps (6-13) for E4M3 data
constexpr int kFp8XformThreads = kThreadsFp8 - 192;
constexpr int kMaxStages = 8;
constexpr int kSmemBudget = 227 * 1024;          // the opt-in maximum per block
constexpr int kBK = 64;                 // K extent of one stage (64 BF16 = 128 B)

struct SmemHeader {
    uint64_t full[kMaxStages];
    uint64_t xform[kMaxStages];     // FP8 data: the stage's BF16 operand is ready
    uint64_t empty[kMaxStages];
    uint64_t tfull[2];
    uint64_t tempty[2];
    uint64_t drain;                 // the MMA thread's completion barrier after an abort
    uint32_t tmem_base;
    int abort;
};

__host__ __device__ inline uint32_t tmem_cols_for(int m_pad) {
    uint32_t need = 2u * (uint32_t)m_pad, c = 32;
    while (c < need) c <<= 1;
    return c;
}

__device__ inline uint8_t* align1024(uint8_t* p) {
    return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

template <int S>
__device__ __forceinline__ void split_store(float y, __nv_bfloat16* dst, int64_t piece_stride) {
    const __nv_bfloat16 h1 = __float2bfloat16_rn(y);
    dst[0] = h1;
    if (S >= 2) {
        const float r1 = y - __bfloat162float(h1);
        const __nv_bfloat16 h2 = __float2bfloat16_rn(r1);
        dst[piece_stride] = h2;
        if (S >= 3) {
            const float r2 = r1 - __bfloat162float(h2);
            dst[2 * piece_stride] = __float2bfloat16_rn(r2);
        }
    }
}

// Common prologue: barriers, TMEM allocation.
__device__ inline void tc_prologue(SmemHeader* hd, int stages, uint32_t tmem_cols, const CUtensorMap* m0,
                                   const CUtensorMap* m1) {
    const int warp = threadIdx.x / 32;
    if (threadIdx.x == 0) {
        for (int i = 0; i < stages; ++i) {
            tc::mbar_init(&hd->full[i], 1);
            tc::mbar_init(&hd->xform[i], kFp8XformThreads);
            tc::mbar_init(&hd->empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&hd->tfull[i], 1);
            tc::mbar_init(&hd->tempty[i], 128);
        }
        tc::mbar_init(&hd->drain, 1);
        hd->abort = 0;
        tc::mbar_init_fence();
        tc::tma_prefetch(m0);
        tc::tma_prefetch(m1);
    }
    if (warp == 1) tc::tmem_alloc(&hd->tmem_base, tmem_cols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

// After an abort the MMA thread (warp 1, lane 0) first waits for its MMAs.
__device__ inline void tc_epilogue_teardown(SmemHeader* hd, uint32_t tmem_cols, int* status) {
    if (threadIdx.x == 32 && *(volatile int*)&hd->abort) tc::drain_mmas(&hd->drain, status);
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x / 32 == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(hd->tmem_base, tmem_cols);
    }
}

// After an abort the producer waits (briefly, bounded) for its last copies.
__device__ inline void drain_copies(SmemHeader* hd, uint32_t issued, int stages, int* status) {
    const uint32_t first = issued > (uint32_t)stages ? issued - (uint32_t)stages : 0u;
    for (uint32_t it = first; it < issued; ++it)
        tc::mbar_wait(&hd->full[it % stages], (it / stages) & 1u, status, 100000000ull);
}

// ---------------------------------------------------------------- FP8 data
//
// E4M3 X is widened to BF16 in shared memory by eight transform warps (6-13):
// every E4M3 value is exact in BF16, so the MMAs see the stored values.  The
// row scale s_r of X = diag(s) X8 is applied in the Y epilogue as s_r^2:
// Z = X^T X V = X8^T diag(s^2) (X8 V), so the Z = X^T Y kernel runs on X8 and
// Y' = diag(s^2) X8 V unchanged.

// Two E4M3 codes (low byte first) -> BF16x2 with the hardware conversions:
// E4M3 -> FP16 (exact), FP16 -> FP32 (exact), FP32 -> BF16 (exact: at most
// four significant bits).
__device__ __forceinline__ uint32_t e4m3x2_to_bf16x2_cvt(uint32_t two) {
    uint32_t h2, out;
    float lo, hi;
    asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(h2) : "h"((unsigned short)two));
    asm("{\n\t.reg .f16 l, h;\n\tmov.b32 {l, h}, %2;\n\tcvt.f32.f16 %0, l;\n\tcvt.f32.f16 %1, h;\n\t}"
        : "=f"(lo), "=f"(hi)
        : "r"(h2));
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(out) : "f"(hi), "f"(lo));
    return out;
}

// 16 E4M3 bytes -> 16 BF16 values (two 16-byte chunks).
__device__ __forceinline__ void widen16(const uint4 raw, uint4& lo, uint4& hi) {
    const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
    uint32_t o[8];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        o[2 * i] = e4m3x2_to_bf16x2_cvt(w[i] & 0xFFFFu);
        o[2 * i + 1] = e4m3x2_to_bf16x2_cvt(w[i] >> 16);
    }
    lo = make_uint4(o[0], o[1], o[2], o[3]);
    hi = make_uint4(o[4], o[5], o[6], o[7]);
}

// ---------------------------------------------------------------- Y = X V

// Split K: with ksplit > 1 a task is (tile t, K-range ks) and writes its FP32
// partial Y rows to Ypart[ks][row][m_pad]; ypart_reduce_kernel sums them and
// splits the sum into the BF16 pieces (for few row tiles and large d, e.g. a
// minibatch of a wide matrix).
// FP8X: X is E4M3 (stage = [raw 128 x 64 bytes][BF16 A][V pieces]), row scales
// `scales` (rows r0.., `rows` valid) applied as s_r^2 to Y.
template <int S, bool FP8X>
__global__ void __launch_bounds__(FP8X ? kThreadsFp8 : kThreads, 1)
    xv_tc_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmV, int ntiles,
                 int nk, int m_pad, int stages, __nv_bfloat16* __restrict__ Yt, int64_t ldy, int ksplit,
                 float* __restrict__ Ypart, const float* __restrict__ scales, int64_t rows, int* status,
                 const int64_t* __restrict__ row0) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* tiles = align1024(smem_raw);
    constexpr uint32_t raw_bytes = FP8X ? 128u * 64u : 0u;
    const uint32_t a_bytes = 128u * 128u;
    const uint32_t b_piece = (uint32_t)m_pad * 128u;
    const uint32_t stage_bytes = raw_bytes + a_bytes + S * b_piece;
    SmemHeader* hd = reinterpret_cast<SmemHeader*>(tiles + (size_t)stages * stage_bytes);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const uint32_t tmem_cols = tmem_cols_for(m_pad);
    tc_prologue(hd, stages, tmem_cols, &tmX, &tmV);
    const uint32_t tmem = hd->tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            const int xr0 = row0 ? (int)*row0 : 0;     // device-side first row of X (graph-replayed steps)
            for (int task = blockIdx.x; task < ntiles * ksplit && ok; task += gridDim.x) {
                const int t = task / ksplit, ks = task % ksplit;
                const int k0 = (int)((int64_t)ks * nk / ksplit), k1 = (int)((int64_t)(ks + 1) * nk / ksplit);
                for (int k = k0; k < k1; ++k, ++it) {
                    const uint32_t s = it % stages, ph = (it / stages) & 1u;
                    if (!tc::mbar_wait(&hd->empty[s], ph ^ 1u, status) || *(volatile int*)&hd->abort) {
                        hd->abort = 1;
                        ok = false;
                        break;
                    }
                    tc::mbar_expect_tx(&hd->full[s], FP8X ? raw_bytes + S * b_piece : stage_bytes);
                    uint8_t* st = tiles + (size_t)s * stage_bytes;
                    tc::tma_load_2d(st, &tmX, &hd->full[s], k * kBK, xr0 + t * 128);
#pragma unroll
                    for (int p = 0; p < S; ++p)
                        tc::tma_load_2d(st + raw_bytes + a_bytes + p * b_piece, &tmV, &hd->full[s], k * kBK,
                                        p * m_pad);
                }
            }
            if (!ok) drain_copies(hd, it, stages, status);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_bf16(128, m_pad, false, false);
            uint32_t it = 0, tl = 0;
            bool ok = true;
            for (int task = blockIdx.x; task < ntiles * ksplit && ok; task += gridDim.x, ++tl) {
                const int ks = task % ksplit;
                const int k0 = (int)((int64_t)ks * nk / ksplit), k1 = (int)((int64_t)(ks + 1) * nk / ksplit);
                const uint32_t b = tl & 1u, tph = (tl >> 1) & 1u;
                if (!tc::mbar_wait(&hd->tempty[b], tph ^ 1u, status) || *(volatile int*)&hd->abort) {
                    hd->abort = 1;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t d_tmem = tmem + b * (uint32_t)m_pad;
                for (int k = k0; k < k1; ++k, ++it) {
                    const uint32_t s = it % stages, ph = (it / stages) & 1u;
                    if (!tc::mbar_wait(FP8X ? &hd->xform[s] : &hd->full[s], ph, status) ||
                        *(volatile int*)&hd->abort) {
                        hd->abort = 1;
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t a_addr = tc::smem_u32(tiles + (size_t)s * stage_bytes + raw_bytes);
#pragma unroll
                    for (int kk = 0; kk < kBK / 16; ++kk) {
                        const uint64_t adesc = tc::smem_desc_sw128(a_addr + kk * 32, 16, 1024);
#pragma unroll
                        for (int p = 0; p < S; ++p) {
                            const uint64_t bdesc =
                                tc::smem_desc_sw128(a_addr + a_bytes + p * b_piece + kk * 32, 16, 1024);
                            tc::mma_f16(d_tmem, adesc, bdesc, idesc, (k != k0 || kk != 0 || p != 0) ? 1u : 0u);
                        }
                    }
                    tc::mma_commit(&hd->empty[s]);
                }
                if (ok) tc::mma_commit(&hd->tfull[b]);
            }
        }
    } else if (warp < 6) {
        const int q = warp & 3;
        uint32_t tl = 0;
        for (int task = blockIdx.x; task < ntiles * ksplit; task += gridDim.x, ++tl) {
            const int t = task / ksplit, ks = task % ksplit;
            const uint32_t b = tl & 1u, tph = (tl >> 1) & 1u;
            if (!tc::mbar_wait(&hd->tfull[b], tph, status) || *(volatile int*)&hd->abort) {
                hd->abort = 1;
                break;
            }
            tc::fence_after_sync();
            const int64_t row = (int64_t)t * 128 + q * 32 + lane;
            float rs = 1.f;
            if (FP8X) {
                const float sr = row < rows ? scales[row] : 0.f;
                rs = sr * sr;
            }
            for (int c0 = 0; c0 < m_pad; c0 += 32) {
                uint32_t r[32];
                tc::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + b * (uint32_t)m_pad + (uint32_t)c0, r);
                tc::tmem_ld_wait();
                if (FP8X) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) r[j] = __float_as_uint(__uint_as_float(r[j]) * rs);
                }
                if (ksplit == 1) {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        split_store<S>(__uint_as_float(r[j]), Yt + (int64_t)(c0 + j) * ldy + row,
                                       (int64_t)m_pad * ldy);
                } else {
                    float4* dst = reinterpret_cast<float4*>(Ypart + ((int64_t)ks * ldy + row) * m_pad + c0);
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        dst[j] = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                                             __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
                }
            }
            tc::fence_before_sync();
            tc::mbar_arrive(&hd->tempty[b]);
        }
    } else if (FP8X) {
        // transform: raw row r (64 bytes, unswizzled) -> BF16 row r of A (128 bytes, 128-byte swizzle);
        // task (r, q): raw bytes 16q..16q+15 -> A chunks 2q, 2q + 1
        const int tid = threadIdx.x - 192;
        uint32_t it = 0;
        bool ok = true;
        for (int task = blockIdx.x; task < ntiles * ksplit && ok; task += gridDim.x) {
            const int ks = task % ksplit;
            const int k0 = (int)((int64_t)ks * nk / ksplit), k1 = (int)((int64_t)(ks + 1) * nk / ksplit);
            for (int k = k0; k < k1; ++k, ++it) {
                const uint32_t s = it % stages, ph = (it / stages) & 1u;
                if (!tc::mbar_wait(&hd->full[s], ph, status) || *(volatile int*)&hd->abort) {
                    hd->abort = 1;
                    ok = false;
                    break;
                }
                uint8_t* st = tiles + (size_t)s * stage_bytes;
#pragma unroll
                for (int i = 0; i < 512 / kFp8XformThreads; ++i) {
                    const int id = i * kFp8XformThreads + tid, r = id >> 2, q = id & 3;
                    const uint4 raw = *reinterpret_cast<const uint4*>(st + r * 64 + q * 16);
                    uint4 lo, hi;
                    widen16(raw, lo, hi);
                    uint8_t* arow = st + raw_bytes + r * 128;
                    *reinterpret_cast<uint4*>(arow + (((2 * q) ^ (r & 7)) << 4)) = lo;
                    *reinterpret_cast<uint4*>(arow + (((2 * q + 1) ^ (r & 7)) << 4)) = hi;
                }
                tc::fence_proxy_async_shared();
                tc::mbar_arrive(&hd->xform[s]);
            }
        }
    }
    tc_epilogue_teardown(hd, tmem_cols, status);
}

// ---------------------------------------------------------------- Z = X^T Y

// FP8X: X is E4M3 (stage = [raw 64 rows x 128 bytes][BF16 A][Y pieces]).
template <int S, bool FP8X>
__global__ void __launch_bounds__(FP8X ? kThreadsFp8 : kThreads, 1)
    xty_tc_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY, int Dt, int Sg,
                  int kst, int flush, int m_pad, int stages, float* __restrict__ Zacc, int* status,
                  const int64_t* __restrict__ row0) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* tiles = align1024(smem_raw);
    constexpr uint32_t raw_bytes = FP8X ? 64u * 128u : 0u;
    const uint32_t a_bytes = 2u * 64u * 128u;     // two 64-row x 64-col boxes
    const uint32_t b_piece = (uint32_t)m_pad * 128u;
    const uint32_t stage_bytes = raw_bytes + a_bytes + S * b_piece;
    SmemHeader* hd = reinterpret_cast<SmemHeader*>(tiles + (size_t)stages * stage_bytes);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const uint32_t tmem_cols = tmem_cols_for(m_pad);
    tc_prologue(hd, stages, tmem_cols, &tmX, &tmY);
    const uint32_t tmem = hd->tmem_base;
    const int ntask = Dt * Sg;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            const int xr0 = row0 ? (int)*row0 : 0;     // device-side first row of X (graph-replayed steps)
            for (int task = blockIdx.x; task < ntask && ok; task += gridDim.x) {
                const int s = task % Dt, g = task / Dt;
                const int k0 = (int)((int64_t)g * kst / Sg), k1 = (int)((int64_t)(g + 1) * kst / Sg);
                for (int k = k0; k < k1; ++k, ++it) {
                    const uint32_t st_i = it % stages, ph = (it / stages) & 1u;
                    if (!tc::mbar_wait(&hd->empty[st_i], ph ^ 1u, status) || *(volatile int*)&hd->abort) {
                        hd->abort = 1;
                        ok = false;
                        break;
                    }
                    tc::mbar_expect_tx(&hd->full[st_i], FP8X ? raw_bytes + S * b_piece : stage_bytes);
                    uint8_t* st = tiles + (size_t)st_i * stage_bytes;
                    tc::tma_load_2d(st, &tmX, &hd->full[st_i], s * 128, xr0 + k * kBK);
                    if (!FP8X) tc::tma_load_2d(st + 8192, &tmX, &hd->full[st_i], s * 128 + 64, xr0 + k * kBK);
#pragma unroll
                    for (int p = 0; p < S; ++p)
                        tc::tma_load_2d(st + raw_bytes + a_bytes + p * b_piece, &tmY, &hd->full[st_i], k * kBK,
                                        p * m_pad);
                }
            }
            if (!ok) drain_copies(hd, it, stages, status);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_bf16(128, m_pad, true, false);
            uint32_t it = 0, fb = 0;
            bool ok = true;
            for (int task = blockIdx.x; task < ntask && ok; task += gridDim.x) {
                const int g = task / Dt;
                const int k0 = (int)((int64_t)g * kst / Sg), k1 = (int)((int64_t)(g + 1) * kst / Sg);
                for (int kb = k0; kb < k1 && ok; kb += flush, ++fb) {
                    const int ke = kb + flush < k1 ? kb + flush : k1;
                    const uint32_t b = fb & 1u, tph = (fb >> 1) & 1u;
                    if (!tc::mbar_wait(&hd->tempty[b], tph ^ 1u, status) || *(volatile int*)&hd->abort) {
                        hd->abort = 1;
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t d_tmem = tmem + b * (uint32_t)m_pad;
                    for (int k = kb; k < ke; ++k, ++it) {
                        const uint32_t st_i = it % stages, ph = (it / stages) & 1u;
                        if (!tc::mbar_wait(FP8X ? &hd->xform[st_i] : &hd->full[st_i], ph, status) ||
                            *(volatile int*)&hd->abort) {
                            hd->abort = 1;
                            ok = false;
                            break;
                        }
                        tc::fence_after_sync();
                        const uint32_t a_addr = tc::smem_u32(tiles + (size_t)st_i * stage_bytes + raw_bytes);
#pragma unroll
                        for (int kk = 0; kk < kBK / 16; ++kk) {
                            const uint64_t adesc = tc::smem_desc_sw128(a_addr + kk * 2048, 8192, 1024);
#pragma unroll
                            for (int p = 0; p < S; ++p) {
                                const uint64_t bdesc =
                                    tc::smem_desc_sw128(a_addr + a_bytes + p * b_piece + kk * 32, 16, 1024);
                                tc::mma_f16(d_tmem, adesc, bdesc, idesc, (k != kb) || kk != 0 || p != 0);
                            }
                        }
                        tc::mma_commit(&hd->empty[st_i]);
                    }
                    if (ok) tc::mma_commit(&hd->tfull[b]);
                }
            }
        }
    } else if (warp < 6) {
        const int q = warp & 3;
        uint32_t fb = 0;
        bool ok = true;
        for (int task = blockIdx.x; task < ntask && ok; task += gridDim.x) {
            const int s = task % Dt, g = task / Dt;
            const int k0 = (int)((int64_t)g * kst / Sg), k1 = (int)((int64_t)(g + 1) * kst / Sg);
            const int64_t j = (int64_t)s * 128 + q * 32 + lane;
            const int64_t zs = (int64_t)Dt * 128;     // Z partials [g][column][row]: a warp's rows contiguous
            float2* z = reinterpret_cast<float2*>(Zacc) + (int64_t)g * m_pad * zs + j;
            for (int kb = k0; kb < k1; kb += flush, ++fb) {
                const uint32_t b = fb & 1u, tph = (fb >> 1) & 1u;
                if (!tc::mbar_wait(&hd->tfull[b], tph, status) || *(volatile int*)&hd->abort) {
                    hd->abort = 1;
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                for (int c0 = 0; c0 < m_pad; c0 += 32) {
                    uint32_t r[32];
                    tc::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + b * (uint32_t)m_pad + (uint32_t)c0, r);
                    tc::tmem_ld_wait();
                    float2* zz = z + (int64_t)c0 * zs;
                    if (kb == k0) {
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj) zz[jj * zs] = make_float2(__uint_as_float(r[jj]), 0.f);
                    } else {
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj) {
                            float2 v = zz[jj * zs];
                            df_add(v.x, v.y, __uint_as_float(r[jj]));
                            zz[jj * zs] = v;
                        }
                    }
                }
                tc::fence_before_sync();
                tc::mbar_arrive(&hd->tempty[b]);
            }
        }
    } else if (FP8X) {
        // transform: raw [64 rows][128 bytes] (columns of the 128-column slice) -> two BF16
        // boxes [64 rows][64 columns] (128-byte swizzle), the MN-major operand X^T;
        // task (r, q): raw bytes 16q..16q+15 -> box q / 4, chunks 2 (q % 4), 2 (q % 4) + 1 of row r
        const int tid = threadIdx.x - 192;
        uint32_t it = 0;
        bool ok = true;
        for (int task = blockIdx.x; task < ntask && ok; task += gridDim.x) {
            const int g = task / Dt;
            const int k0 = (int)((int64_t)g * kst / Sg), k1 = (int)((int64_t)(g + 1) * kst / Sg);
            for (int k = k0; k < k1; ++k, ++it) {
                const uint32_t st_i = it % stages, ph = (it / stages) & 1u;
                if (!tc::mbar_wait(&hd->full[st_i], ph, status) || *(volatile int*)&hd->abort) {
                    hd->abort = 1;
                    ok = false;
                    break;
                }
                uint8_t* st = tiles + (size_t)st_i * stage_bytes;
#pragma unroll
                for (int i = 0; i < 512 / kFp8XformThreads; ++i) {
                    const int id = i * kFp8XformThreads + tid, r = id >> 3, q = id & 7;
                    const uint4 raw = *reinterpret_cast<const uint4*>(st + r * 128 + q * 16);
                    uint4 lo, hi;
                    widen16(raw, lo, hi);
                    uint8_t* arow = st + raw_bytes + (q >> 2) * 8192 + r * 128;
                    const int c = 2 * (q & 3);
                    // lanes q and q + 4 write the same row of the two boxes (8 KB apart, the
                    // same banks): the second box stores its odd chunk first, so the eight
                    // lanes of each 16-byte store phase touch eight different chunks
                    // (selects, not a branch: each store stays one instruction for the warp)
                    const bool first_box = q < 4;
                    const int c1 = first_box ? c : c + 1, c2 = first_box ? c + 1 : c;
                    *reinterpret_cast<uint4*>(arow + ((c1 ^ (r & 7)) << 4)) = first_box ? lo : hi;
                    *reinterpret_cast<uint4*>(arow + ((c2 ^ (r & 7)) << 4)) = first_box ? hi : lo;
                }
                tc::fence_proxy_async_shared();
                tc::mbar_arrive(&hd->xform[st_i]);
            }
        }
    }
    tc_epilogue_teardown(hd, tmem_cols, status);
}

// ---------------------------------------------------------------- FP8 data on kind::f8f6f4
//
// The FAST pass of E4M3 data straight on the FP8 tensor cores, with no
// widening: X8 (the stored codes) is the A operand as loaded.  V and Y enter
// as two E4M3 pieces that share one power-of-two scale, hi = E4M3(2^a v) and
// lo = E4M3(2^a v - hi), so both pieces' MMAs accumulate into one FP32
// accumulator: X8 (hi + lo) = 2^a X8 V with about 2^-8 relative error per term
// (a value below 2^-10 of the scaled range keeps an absolute error under
// 2^-17 of the range).  With X = diag(s) X8,
//   Y' = diag(s^2) X8 V    (rows r0..r1; xv_f8_kernel, pieces at scale 2^b)
//   Z  = X8^T Y'           (xty_f8_kernel; X8^T read MN-major)
// The scales come from three maxima taken before the pass (f8_stats_kernel):
// 2^a is the largest power of two with max|V| 2^a <= 448, and 2^b the largest
// with sqrt(d) max_r s_r^2 max_c |v_c| 2^b <= 1, a bound on |Y'| / 448 since
// |x8_r . v_c| <= |x8_r| |v_c| <= 448 sqrt(d) |v_c|.  f8s[] holds
// {max|V|, max_c |v_c|^2, max_r s_r^2, 2^(b - a), 2^-b}.

// (e4m3(hi_elem) << 8) | e4m3(lo_elem), round to nearest even, saturating at 448.
__device__ __forceinline__ uint32_t f32x2_to_e4m3x2(float hi_elem, float lo_elem) {
    uint16_t r;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(r) : "f"(hi_elem), "f"(lo_elem));
    return r;
}

// Two E4M3 codes (low byte -> .x, high byte -> .y) as exact FP32 values.
__device__ __forceinline__ float2 e4m3x2_to_f32x2(uint32_t two) {
    uint32_t h2;
    float lo, hi;
    asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(h2) : "h"((unsigned short)two));
    asm("{\n\t.reg .f16 l, h;\n\tmov.b32 {l, h}, %2;\n\tcvt.f32.f16 %0, l;\n\tcvt.f32.f16 %1, h;\n\t}"
        : "=f"(lo), "=f"(hi)
        : "r"(h2));
    return make_float2(lo, hi);
}

// Two values -> their hi and lo E4M3 pieces (each a code pair, low byte = y0).
__device__ __forceinline__ void e4m3_pieces(float y0, float y1, uint32_t& hi, uint32_t& lo) {
    hi = f32x2_to_e4m3x2(y1, y0);
    const float2 b = e4m3x2_to_f32x2(hi);
    lo = f32x2_to_e4m3x2(y1 - b.y, y0 - b.x);
}

// Largest power of two p with p * v <= cap (v > 0), as a float; 1 for v == 0.
__device__ __forceinline__ float pow2_below(float cap, float v) {
    if (!(v > 0.f)) return 1.f;
    int e;
    frexpf(cap / v, &e);                       // cap / v = f 2^e, f in [0.5, 1)
    e = e - 1;
    e = e < -126 ? -126 : (e > 126 ? 126 : e);
    return ldexpf(1.f, e);
}

__device__ __forceinline__ void atomic_max_nonneg(float* p, float v) {
    atomicMax(reinterpret_cast<int*>(p), __float_as_int(v));   // non-negative floats order as their bits
}

// Blocks 0..m-1: column c of V (max |v_kc| and |v_c|^2); the rest: max s_r^2 over rows [0, rows).
__global__ void f8_stats_kernel(const float* __restrict__ V, int64_t d, int m, const float* __restrict__ scales,
                                int64_t rows, float* __restrict__ f8s) {
    __shared__ float red[2][32];
    float a = 0.f, q = 0.f;
    if ((int)blockIdx.x < m) {
        const float* v = V + (int64_t)blockIdx.x * d;
        for (int64_t k = threadIdx.x; k < d; k += blockDim.x) {
            const float x = v[k];
            a = fmaxf(a, fabsf(x));
            q = fmaf(x, x, q);
        }
    } else {
        for (int64_t r = (int64_t)(blockIdx.x - m) * blockDim.x + threadIdx.x; r < rows;
             r += (int64_t)(gridDim.x - m) * blockDim.x) {
            const float sr = scales[r];
            a = fmaxf(a, sr * sr);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
        q += __shfl_xor_sync(0xffffffffu, q, o);
    }
    const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (lane == 0) {
        red[0][w] = a;
        red[1][w] = q;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x / 32); ++i) {
            a = fmaxf(a, red[0][i]);
            q += red[1][i];
        }
        if ((int)blockIdx.x < m) {
            atomic_max_nonneg(&f8s[0], a);
            atomic_max_nonneg(&f8s[1], q);
        } else {
            atomic_max_nonneg(&f8s[2], a);
        }
    }
}

// V (d x m column-major FP32) -> hi and lo E4M3 pieces at the shared scale 2^a,
// [2][m_pad][ldv8] bytes, zero padded; thread (0, 0) also stores 2^(b - a) and 2^-b.
__global__ void split_v8_kernel(const float* __restrict__ V, int64_t d, int m, int m_pad, int64_t ldv8,
                                float* __restrict__ f8s, uint8_t* __restrict__ V8) {
    const float sa = pow2_below(448.f, f8s[0]);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const float bound = sqrtf((float)d) * f8s[2] * sqrtf(f8s[1]);
        const float sb = pow2_below(1.f, bound);
        f8s[3] = sb / sa;
        f8s[4] = 1.f / sb;
    }
    const int64_t pairs = (int64_t)m_pad * ldv8 / 2;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < pairs; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / (ldv8 / 2), k = (e % (ldv8 / 2)) * 2;
        const float v0 = (c < m && k < d) ? V[c * d + k] * sa : 0.f;
        const float v1 = (c < m && k + 1 < d) ? V[c * d + k + 1] * sa : 0.f;
        uint32_t hi, lo;
        e4m3_pieces(v0, v1, hi, lo);
        reinterpret_cast<uint16_t*>(V8)[e] = (uint16_t)hi;
        reinterpret_cast<uint16_t*>(V8 + (int64_t)m_pad * ldv8)[e] = (uint16_t)lo;
    }
}

// Y' = diag(s^2) X8 V for 256-row tiles, two M = 128 accumulators sharing each V stage (stage =
// [X8 rows 0-127][X8 rows 128-255][V hi][V lo], 128 B of K each), so a CTA ingests one byte of V pieces
// per byte of X; Y' stored as its hi and lo E4M3 pieces at scale 2^b, Y^T layout [2][m_pad][ldy] bytes
// (ldy a multiple of 256).
__global__ void __launch_bounds__(kThreads, 1)
    xv_f8_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmV, int ntiles,
                 int nk, int m_pad, int stages, uint8_t* __restrict__ Yt, int64_t ldy,
                 const float* __restrict__ scales, int64_t rows, const float* __restrict__ f8s, int* status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* tiles = align1024(smem_raw);
    const uint32_t a_bytes = 2u * 128u * 128u;
    const uint32_t b_piece = (uint32_t)m_pad * 128u;
    const uint32_t stage_bytes = a_bytes + 2u * b_piece;
    SmemHeader* hd = reinterpret_cast<SmemHeader*>(tiles + (size_t)stages * stage_bytes);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const uint32_t tmem_cols = tmem_cols_for(2 * m_pad);      // 2 buffers x 2 row halves
    tc_prologue(hd, stages, tmem_cols, &tmX, &tmV);
    const uint32_t tmem = hd->tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                for (int k = 0; k < nk; ++k, ++it) {
                    const uint32_t s = it % stages, ph = (it / stages) & 1u;
                    if (!tc::mbar_wait(&hd->empty[s], ph ^ 1u, status) || *(volatile int*)&hd->abort) {
                        hd->abort = 1;
                        ok = false;
                        break;
                    }
                    tc::mbar_expect_tx(&hd->full[s], stage_bytes);
                    uint8_t* st = tiles + (size_t)s * stage_bytes;
                    tc::tma_load_2d(st, &tmX, &hd->full[s], k * 128, t * 256);
                    tc::tma_load_2d(st + 16384, &tmX, &hd->full[s], k * 128, t * 256 + 128);
                    tc::tma_load_2d(st + a_bytes, &tmV, &hd->full[s], k * 128, 0);
                    tc::tma_load_2d(st + a_bytes + b_piece, &tmV, &hd->full[s], k * 128, m_pad);
                }
            }
            if (!ok) drain_copies(hd, it, stages, status);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_e4m3(128, m_pad, false, false);
            uint32_t it = 0, tl = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++tl) {
                const uint32_t b = tl & 1u, tph = (tl >> 1) & 1u;
                if (!tc::mbar_wait(&hd->tempty[b], tph ^ 1u, status) || *(volatile int*)&hd->abort) {
                    hd->abort = 1;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t d_tmem = tmem + b * 2u * (uint32_t)m_pad;
                for (int k = 0; k < nk; ++k, ++it) {
                    const uint32_t s = it % stages, ph = (it / stages) & 1u;
                    if (!tc::mbar_wait(&hd->full[s], ph, status) || *(volatile int*)&hd->abort) {
                        hd->abort = 1;
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t a_addr = tc::smem_u32(tiles + (size_t)s * stage_bytes);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
                        for (int p = 0; p < 2; ++p) {
                            const uint64_t bdesc =
                                tc::smem_desc_sw128(a_addr + a_bytes + p * b_piece + kk * 32, 16, 1024);
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const uint64_t adesc = tc::smem_desc_sw128(a_addr + h * 16384 + kk * 32, 16, 1024);
                                tc::mma_f8(d_tmem + h * (uint32_t)m_pad, adesc, bdesc, idesc,
                                           (k != 0 || kk != 0 || p != 0) ? 1u : 0u);
                            }
                        }
                    }
                    tc::mma_commit(&hd->empty[s]);
                }
                if (ok) tc::mma_commit(&hd->tfull[b]);
            }
        }
    } else {
        const int q = warp & 3;
        const float f = f8s[3];                   // 2^(b - a)
        uint32_t tl = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++tl) {
            const uint32_t b = tl & 1u, tph = (tl >> 1) & 1u;
            if (!tc::mbar_wait(&hd->tfull[b], tph, status) || *(volatile int*)&hd->abort) {
                hd->abort = 1;
                break;
            }
            tc::fence_after_sync();
            for (int h = 0; h < 2; ++h) {
                const int64_t row = (int64_t)t * 256 + h * 128 + q * 32 + lane;
                const float sr = row < rows ? scales[row] : 0.f;
                const float rs = sr * sr * f;
                const uint32_t acc = tmem + ((uint32_t)(q * 32) << 16) + (b * 2u + h) * (uint32_t)m_pad;
                for (int c0 = 0; c0 < m_pad; c0 += 32) {
                    uint32_t r[32];
                    tc::tmem_ld32(acc + (uint32_t)c0, r);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 32; j += 2) {
                        uint32_t hi, lo;
                        e4m3_pieces(__uint_as_float(r[j]) * rs, __uint_as_float(r[j + 1]) * rs, hi, lo);
                        uint8_t* y = Yt + (int64_t)(c0 + j) * ldy + row;
                        y[0] = (uint8_t)(hi & 0xFFu);
                        y[ldy] = (uint8_t)(hi >> 8);
                        y[(int64_t)m_pad * ldy] = (uint8_t)(lo & 0xFFu);
                        y[(int64_t)m_pad * ldy + ldy] = (uint8_t)(lo >> 8);
                    }
                }
            }
            tc::fence_before_sync();
            tc::mbar_arrive(&hd->tempty[b]);
        }
    }
    tc_epilogue_teardown(hd, tmem_cols, status);
}

// Z = X8^T Y' for (256-column slice, row group) tasks: two M = 128 accumulators share each Y' stage
// (stage = [X8 128 rows x columns 0-127, MN-major][columns 128-255][Y' hi][Y' lo]); each FP32
// accumulator is folded, times 2^-b, into double-float partials [g][column][Dt2 * 256 rows of Z].
__global__ void __launch_bounds__(kThreads, 1)
    xty_f8_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY, int Dt2, int Sg,
                  int kst, int flush, int m_pad, int stages, float* __restrict__ Zacc, const float* __restrict__ f8s,
                  int* status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* tiles = align1024(smem_raw);
    const uint32_t a_bytes = 2u * 128u * 128u;
    const uint32_t b_piece = (uint32_t)m_pad * 128u;
    const uint32_t stage_bytes = a_bytes + 2u * b_piece;
    SmemHeader* hd = reinterpret_cast<SmemHeader*>(tiles + (size_t)stages * stage_bytes);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const uint32_t tmem_cols = tmem_cols_for(2 * m_pad);      // 2 buffers x 2 column halves
    tc_prologue(hd, stages, tmem_cols, &tmX, &tmY);
    const uint32_t tmem = hd->tmem_base;
    const int ntask = Dt2 * Sg;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            for (int task = blockIdx.x; task < ntask && ok; task += gridDim.x) {
                const int s = task % Dt2, g = task / Dt2;
                const int k0 = (int)((int64_t)g * kst / Sg), k1 = (int)((int64_t)(g + 1) * kst / Sg);
                for (int k = k0; k < k1; ++k, ++it) {
                    const uint32_t st_i = it % stages, ph = (it / stages) & 1u;
                    if (!tc::mbar_wait(&hd->empty[st_i], ph ^ 1u, status) || *(volatile int*)&hd->abort) {
                        hd->abort = 1;
                        ok = false;
                        break;
                    }
                    tc::mbar_expect_tx(&hd->full[st_i], stage_bytes);
                    uint8_t* st = tiles + (size_t)st_i * stage_bytes;
                    tc::tma_load_2d(st, &tmX, &hd->full[st_i], s * 256, k * 128);
                    tc::tma_load_2d(st + 16384, &tmX, &hd->full[st_i], s * 256 + 128, k * 128);
                    tc::tma_load_2d(st + a_bytes, &tmY, &hd->full[st_i], k * 128, 0);
                    tc::tma_load_2d(st + a_bytes + b_piece, &tmY, &hd->full[st_i], k * 128, m_pad);
                }
            }
            if (!ok) drain_copies(hd, it, stages, status);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_e4m3(128, m_pad, true, false);
            uint32_t it = 0, fb = 0;
            bool ok = true;
            for (int task = blockIdx.x; task < ntask && ok; task += gridDim.x) {
                const int g = task / Dt2;
                const int k0 = (int)((int64_t)g * kst / Sg), k1 = (int)((int64_t)(g + 1) * kst / Sg);
                for (int kb = k0; kb < k1 && ok; kb += flush, ++fb) {
                    const int ke = kb + flush < k1 ? kb + flush : k1;
                    const uint32_t b = fb & 1u, tph = (fb >> 1) & 1u;
                    if (!tc::mbar_wait(&hd->tempty[b], tph ^ 1u, status) || *(volatile int*)&hd->abort) {
                        hd->abort = 1;
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t d_tmem = tmem + b * 2u * (uint32_t)m_pad;
                    for (int k = kb; k < ke; ++k, ++it) {
                        const uint32_t st_i = it % stages, ph = (it / stages) & 1u;
                        if (!tc::mbar_wait(&hd->full[st_i], ph, status) || *(volatile int*)&hd->abort) {
                            hd->abort = 1;
                            ok = false;
                            break;
                        }
                        tc::fence_after_sync();
                        const uint32_t a_addr = tc::smem_u32(tiles + (size_t)st_i * stage_bytes);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
                            for (int p = 0; p < 2; ++p) {
                                const uint64_t bdesc =
                                    tc::smem_desc_sw128(a_addr + a_bytes + p * b_piece + kk * 32, 16, 1024);
#pragma unroll
                                for (int h = 0; h < 2; ++h) {
                                    // 32 rows of the MN-major X8 half tile (four 8-row groups of 1 KB)
                                    const uint64_t adesc =
                                        tc::smem_desc_sw128(a_addr + h * 16384 + kk * 4096, 16384, 1024);
                                    tc::mma_f8(d_tmem + h * (uint32_t)m_pad, adesc, bdesc, idesc,
                                               (k != kb) || kk != 0 || p != 0);
                                }
                            }
                        }
                        tc::mma_commit(&hd->empty[st_i]);
                    }
                    if (ok) tc::mma_commit(&hd->tfull[b]);
                }
            }
        }
    } else {
        const int q = warp & 3;
        const float zs_f = f8s[4];                // 2^-b
        uint32_t fb = 0;
        bool ok = true;
        for (int task = blockIdx.x; task < ntask && ok; task += gridDim.x) {
            const int s = task % Dt2, g = task / Dt2;
            const int k0 = (int)((int64_t)g * kst / Sg), k1 = (int)((int64_t)(g + 1) * kst / Sg);
            const int64_t zs = (int64_t)Dt2 * 256;    // Z partials [g][column][row]: a warp's rows contiguous
            for (int kb = k0; kb < k1; kb += flush, ++fb) {
                const uint32_t b = fb & 1u, tph = (fb >> 1) & 1u;
                if (!tc::mbar_wait(&hd->tfull[b], tph, status) || *(volatile int*)&hd->abort) {
                    hd->abort = 1;
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                for (int h = 0; h < 2; ++h) {
                    const int64_t j = (int64_t)s * 256 + h * 128 + q * 32 + lane;
                    float2* z = reinterpret_cast<float2*>(Zacc) + (int64_t)g * m_pad * zs + j;
                    const uint32_t acc = tmem + ((uint32_t)(q * 32) << 16) + (b * 2u + h) * (uint32_t)m_pad;
                    for (int c0 = 0; c0 < m_pad; c0 += 32) {
                        uint32_t r[32];
                        tc::tmem_ld32(acc + (uint32_t)c0, r);
                        tc::tmem_ld_wait();
                        float2* zz = z + (int64_t)c0 * zs;
                        if (kb == k0) {
#pragma unroll
                            for (int jj = 0; jj < 32; ++jj)
                                zz[jj * zs] = make_float2(__uint_as_float(r[jj]) * zs_f, 0.f);
                        } else {
#pragma unroll
                            for (int jj = 0; jj < 32; ++jj) {
                                float2 v = zz[jj * zs];
                                df_add(v.x, v.y, __uint_as_float(r[jj]) * zs_f);
                                zz[jj * zs] = v;
                            }
                        }
                    }
                }
                tc::fence_before_sync();
                tc::mbar_arrive(&hd->tempty[b]);
            }
        }
    }
    tc_epilogue_teardown(hd, tmem_cols, status);
}

// ---------------------------------------------------------------- fused single-read pass
//
// One persistent, cooperatively launched kernel; every CTA runs two
// warp-specialised pipelines that share the tensor core and TMEM:
//   producer (warps 0-5)   Y_t = X_t V for 128-row tiles (X streamed from
//                          HBM), Y_t written as BF16, then ready[t] released
//                          (one add per epilogue warp).  With kparts = 2 a
//                          tile is two work items, the two halves of the K
//                          range (d), taken by neighbouring CTAs: the first
//                          epilogue warp of a row quarter to finish stores
//                          its FP32 partial and releases pready, the second
//                          adds it to its own accumulator and publishes
//                          Y_t.  Half-tiles halve the X bytes in flight
//                          (152 x 0.5 MB instead of 152 x 1 MB), so more
//                          of the consumers' re-reads still find X_t in
//                          L2, at the same V traffic per byte of X;
//   consumer (warps 6-11)  CTA (sp, g) owns the 256-column slice pair sp of Z
//                          for the whole pass (two M = 128 accumulators in
//                          TMEM) and consumes the tiles t = g, g + Sg, ...: it
//                          acquires ready[t] and reads X_t[:, pair] and Y_t --
//                          X_t was loaded by its producer moments earlier, so
//                          the re-read hits L2 -- then counts consumed[t].
// A producer starts tile t only when tile t - window has been consumed by all
// Dt2 slice-pair owners (a guard against runaway, set above the producer
// count).  All waits are bounded (kDevWaitTimeout).
struct FusedHeader {
    uint64_t pfull[kMaxStages], pempty[kMaxStages], ptfull[2], ptempty[2];
    uint64_t cfull[kMaxStages], cempty[kMaxStages], ctfull, ctempty;
    uint64_t pdrain, cdrain;        // the two MMA threads' completion barriers after an abort
    uint32_t tmem_base;
    int abort;
};

constexpr int kFusedThreads = 384;

__global__ void __launch_bounds__(kFusedThreads, 1)
    xpass_fused_kernel(const __grid_constant__ CUtensorMap tmXa, const __grid_constant__ CUtensorMap tmV,
                       const __grid_constant__ CUtensorMap tmXb, const __grid_constant__ CUtensorMap tmY, int ntiles,
                       int nk, int Dt2, int Sg, int NP, int window, int flush_tiles, int m_pad, int p_stages,
                       int c_stages, __nv_bfloat16* __restrict__ Yt, int64_t ldy, float* __restrict__ Zacc,
                       int* __restrict__ ready, int* __restrict__ consumed, int kparts, float* __restrict__ Ypart,
                       int* __restrict__ arrive, int* __restrict__ pready, int kkeep, int* status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* tiles = align1024(smem_raw);
    const uint32_t p_a = 128u * 128u;            // 128 rows x 64 columns
    const int nitems = ntiles * kparts;          // producer work items (tile, K part)
    const int kh = (nk + 1) / 2;                 // K-stages of the first half when kparts = 2
    const uint32_t c_a = 4u * 64u * 128u;        // 64 rows x 256 columns, four 64-column boxes
    const uint32_t b_piece = (uint32_t)m_pad * 128u;
    const uint32_t p_stage = p_a + b_piece, c_stage = c_a + b_piece;
    uint8_t* ptiles = tiles;
    uint8_t* ctiles = tiles + (size_t)p_stages * p_stage;
    FusedHeader* hd = reinterpret_cast<FusedHeader*>(ctiles + (size_t)c_stages * c_stage);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) {
        for (int i = 0; i < p_stages; ++i) {
            tc::mbar_init(&hd->pfull[i], 1);
            tc::mbar_init(&hd->pempty[i], 1);
        }
        for (int i = 0; i < c_stages; ++i) {
            tc::mbar_init(&hd->cfull[i], 1);
            tc::mbar_init(&hd->cempty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&hd->ptfull[i], 1);
            tc::mbar_init(&hd->ptempty[i], 128);
        }
        tc::mbar_init(&hd->ctfull, 1);
        tc::mbar_init(&hd->ctempty, 128);
        tc::mbar_init(&hd->pdrain, 1);
        tc::mbar_init(&hd->cdrain, 1);
        hd->abort = 0;
        tc::mbar_init_fence();
        tc::tma_prefetch(&tmXa);
        tc::tma_prefetch(&tmV);
        tc::tma_prefetch(&tmXb);
        tc::tma_prefetch(&tmY);
    }
    if (warp == 1) tc::tmem_alloc(&hd->tmem_base, 512);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = hd->tmem_base;
    const uint32_t ptmem = tmem, ctmem = tmem + 2u * (uint32_t)m_pad;
    const bool producer = (int)blockIdx.x < NP;
    const int task = blockIdx.x;
    const bool consumer = task < Dt2 * Sg;
    const int sp = consumer ? task % Dt2 : 0, cg = consumer ? task / Dt2 : 0;
    volatile int* abort_flag = &hd->abort;

    if (warp == 0) {
        // ---------------- producer TMA
        if (lane == 0 && producer) {
            // The last K-stages of every tile (k >= kkeep) are loaded evict_last, so
            // they stay in L2 until the consumers re-read them (evict_first there);
            // the first ones are loaded evict_first.  All 152 tiles in flight
            // would not fit in L2: protecting all of them lets the oldest parts
            // of every tile evict one another, protecting a part that fits keeps it.
            const uint64_t keep = tc::policy_evict_last(), drop_early = tc::policy_evict_first();
            uint32_t it = 0;
            bool ok = true;
            for (int i = blockIdx.x; i < nitems && ok; i += NP) {
                const int t = i / kparts, part = i - t * kparts;
                const int kb0 = part ? kh : 0, kb1 = (kparts == 1 || part) ? nk : kh;
                if (t >= window && !tc::wait_flag_geq(consumed + (t - window), Dt2, status)) {
                    *abort_flag = 1;
                    break;
                }
                for (int k = kb0; k < kb1; ++k, ++it) {
                    const uint32_t s = it % p_stages, ph = (it / p_stages) & 1u;
                    if (!tc::mbar_wait(&hd->pempty[s], ph ^ 1u, status) || *abort_flag) {
                        *abort_flag = 1;
                        ok = false;
                        break;
                    }
                    tc::mbar_expect_tx(&hd->pfull[s], p_stage);
                    uint8_t* st = ptiles + (size_t)s * p_stage;
                    tc::tma_load_2d_hint(st, &tmXa, &hd->pfull[s], k * kBK, t * 128, k >= kkeep ? keep : drop_early);
                    tc::tma_load_2d(st + p_a, &tmV, &hd->pfull[s], k * kBK, 0);
                }
            }
            const uint32_t first = it > (uint32_t)p_stages ? it - (uint32_t)p_stages : 0u;
            if (*abort_flag)
                for (uint32_t j = first; j < it; ++j)
                    tc::mbar_wait(&hd->pfull[j % p_stages], (j / p_stages) & 1u, status, 100000000ull);
        }
    } else if (warp == 1) {
        // ---------------- producer MMA
        if (lane == 0 && producer) {
            const uint32_t idesc = tc::idesc_bf16(128, m_pad, false, false);
            uint32_t it = 0, tl = 0;
            bool ok = true;
            for (int i = blockIdx.x; i < nitems && ok; i += NP, ++tl) {
                const int part = i % kparts;
                const int kb0 = part ? kh : 0, kb1 = (kparts == 1 || part) ? nk : kh;
                const uint32_t b = tl & 1u, tph = (tl >> 1) & 1u;
                if (!tc::mbar_wait(&hd->ptempty[b], tph ^ 1u, status) || *abort_flag) {
                    *abort_flag = 1;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t d_tmem = ptmem + b * (uint32_t)m_pad;
                for (int k = kb0; k < kb1; ++k, ++it) {
                    const uint32_t s = it % p_stages, ph = (it / p_stages) & 1u;
                    if (!tc::mbar_wait(&hd->pfull[s], ph, status) || *abort_flag) {
                        *abort_flag = 1;
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t a_addr = tc::smem_u32(ptiles + (size_t)s * p_stage);
#pragma unroll
                    for (int kk = 0; kk < kBK / 16; ++kk) {
                        const uint64_t adesc = tc::smem_desc_sw128(a_addr + kk * 32, 16, 1024);
                        const uint64_t bdesc = tc::smem_desc_sw128(a_addr + p_a + kk * 32, 16, 1024);
                        tc::mma_f16(d_tmem, adesc, bdesc, idesc, (k - kb0 | kk) != 0);
                    }
                    tc::mma_commit(&hd->pempty[s]);
                }
                if (ok) tc::mma_commit(&hd->ptfull[b]);
            }
        }
    } else if (warp < 6) {
        // ---------------- producer epilogue: Y_t -> BF16, then release ready[t]
        if (producer) {
            const int q = warp & 3;
            uint32_t tl = 0;
            for (int i = blockIdx.x; i < nitems; i += NP, ++tl) {
                const int t = i / kparts;
                const uint32_t b = tl & 1u, tph = (tl >> 1) & 1u;
                if (!tc::mbar_wait(&hd->ptfull[b], tph, status) || *abort_flag) {
                    *abort_flag = 1;
                    break;
                }
                tc::fence_after_sync();
                const int64_t row = (int64_t)t * 128 + q * 32 + lane;
                const uint32_t acc = ptmem + ((uint32_t)(q * 32) << 16) + b * (uint32_t)m_pad;
                // partial of this row quarter: [tile][column][128 rows] FP32, one 128-byte line per column
                float* yp = Ypart + ((int64_t)t * m_pad) * 128 + q * 32;
                int order = 1;                                   // kparts = 1: the only (= last) arrival
                if (kparts == 2) {
                    if (lane == 0) order = atomicAdd(arrive + t * 4 + q, 1);
                    order = __shfl_sync(0xffffffffu, order, 0);
                }
                if (order == 0) {
                    // first half done: store the FP32 partial, then release it
                    for (int c0 = 0; c0 < m_pad; c0 += 32) {
                        uint32_t r[32];
                        tc::tmem_ld32(acc + (uint32_t)c0, r);
                        tc::tmem_ld_wait();
#pragma unroll
                        for (int j = 0; j < 32; ++j) yp[(int64_t)(c0 + j) * 128 + lane] = __uint_as_float(r[j]);
                    }
                    tc::fence_before_sync();
                    tc::mbar_arrive(&hd->ptempty[b]);
                    __threadfence();
                    __syncwarp();
                    if (lane == 0) tc::red_release_add_gpu(pready + t * 4 + q, 1);
                    continue;
                }
                if (kparts == 2 && (!tc::wait_flag_geq(pready + t * 4 + q, 1, status) || *abort_flag)) {
                    *abort_flag = 1;
                    break;
                }
                for (int c0 = 0; c0 < m_pad; c0 += 32) {
                    uint32_t r[32];
                    tc::tmem_ld32(acc + (uint32_t)c0, r);
                    tc::tmem_ld_wait();
                    if (kparts == 2) {
                        // FP32 a + b is commutative: Y_t does not depend on which half came first
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            r[j] = __float_as_uint(__uint_as_float(r[j]) + __ldcg(yp + (int64_t)(c0 + j) * 128 + lane));
                    }
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        Yt[(int64_t)(c0 + j) * ldy + row] = __float2bfloat16_rn(__uint_as_float(r[j]));
                }
                tc::fence_before_sync();
                tc::mbar_arrive(&hd->ptempty[b]);
                if (kparts == 2) {
                    // the partial is dead: drop its lines from L2 without writing them back
                    __syncwarp();
                    for (int c = lane; c < m_pad; c += 32) tc::discard_l2_line(yp + (int64_t)c * 128);
                }
                // publish: every lane fences its stores, the warp syncs, and one
                // lane adds a release to ready[t]; consumers wait for all 4 warps
                __threadfence();
                __syncwarp();
                if (lane == 0) tc::red_release_add_gpu(ready + t, 1);
            }
        }
    } else if (warp == 6) {
        // ---------------- consumer TMA
        if (lane == 0 && consumer) {
            const uint64_t drop = tc::policy_evict_first();
            uint32_t it = 0;
            bool ok = true;
            for (int t = cg; t < ntiles && ok; t += Sg) {
                if (!tc::wait_flag_geq(ready + t, 4, status) || *abort_flag) {
                    *abort_flag = 1;
                    break;
                }
                tc::fence_proxy_async_global();
                for (int kk2 = 0; kk2 < 2; ++kk2, ++it) {
                    const uint32_t s = it % c_stages, ph = (it / c_stages) & 1u;
                    if (!tc::mbar_wait(&hd->cempty[s], ph ^ 1u, status) || *abort_flag) {
                        *abort_flag = 1;
                        ok = false;
                        break;
                    }
                    tc::mbar_expect_tx(&hd->cfull[s], c_stage);
                    uint8_t* st = ctiles + (size_t)s * c_stage;
                    const int y = t * 128 + kk2 * 64;
#pragma unroll
                    for (int bx = 0; bx < 4; ++bx)
                        tc::tma_load_2d_hint(st + bx * 8192, &tmXb, &hd->cfull[s], sp * 256 + bx * 64, y, drop);
                    tc::tma_load_2d(st + c_a, &tmY, &hd->cfull[s], y, 0);
                }
            }
            const uint32_t first = it > (uint32_t)c_stages ? it - (uint32_t)c_stages : 0u;
            if (*abort_flag)
                for (uint32_t j = first; j < it; ++j)
                    tc::mbar_wait(&hd->cfull[j % c_stages], (j / c_stages) & 1u, status, 100000000ull);
        }
    } else if (warp == 7) {
        // ---------------- consumer MMA: Z[pair] accumulates across tiles, two M = 128 halves
        if (lane == 0 && consumer) {
            const uint32_t idesc = tc::idesc_bf16(128, m_pad, true, false);
            uint32_t it = 0, fb = 0;
            bool ok = true;
            int t = cg;
            while (t < ntiles && ok) {
                if (!tc::mbar_wait(&hd->ctempty, (fb & 1u) ^ 1u, status) || *abort_flag) {
                    *abort_flag = 1;
                    break;
                }
                tc::fence_after_sync();
                for (int nt = 0; nt < flush_tiles && t < ntiles && ok; ++nt, t += Sg) {
                    for (int kk2 = 0; kk2 < 2; ++kk2, ++it) {
                        const uint32_t s = it % c_stages, ph = (it / c_stages) & 1u;
                        if (!tc::mbar_wait(&hd->cfull[s], ph, status) || *abort_flag) {
                            *abort_flag = 1;
                            ok = false;
                            break;
                        }
                        tc::fence_after_sync();
                        const uint32_t a_addr = tc::smem_u32(ctiles + (size_t)s * c_stage);
#pragma unroll
                        for (int kk = 0; kk < kBK / 16; ++kk) {
                            const uint64_t bdesc = tc::smem_desc_sw128(a_addr + c_a + kk * 32, 16, 1024);
#pragma unroll
                            for (int hh = 0; hh < 2; ++hh) {
                                const uint64_t adesc =
                                    tc::smem_desc_sw128(a_addr + hh * 16384 + kk * 2048, 8192, 1024);
                                tc::mma_f16(ctmem + hh * (uint32_t)m_pad, adesc, bdesc, idesc, (nt | kk2 | kk) != 0);
                            }
                        }
                        tc::mma_commit(&hd->cempty[s]);
                    }
                    if (ok) atomicAdd(consumed + t, 1);     // tile t's column pair has been read
                }
                if (ok) tc::mma_commit(&hd->ctfull);
                ++fb;
            }
        }
    } else {
        // ---------------- consumer epilogue: fold the block sums into the double-float partials
        if (consumer) {
            const int q = warp & 3;
            uint32_t fb = 0;
            for (int t = cg; t < ntiles; t += Sg * flush_tiles, ++fb) {
                if (!tc::mbar_wait(&hd->ctfull, fb & 1u, status) || *abort_flag) {
                    *abort_flag = 1;
                    break;
                }
                tc::fence_after_sync();
                for (int hh = 0; hh < 2; ++hh) {
                    const int64_t j = (int64_t)sp * 256 + hh * 128 + q * 32 + lane;
                    const int64_t zs = (int64_t)Dt2 * 256;   // Z partials [g][column][row]: a warp's rows contiguous
                    float2* z = reinterpret_cast<float2*>(Zacc) + (int64_t)cg * m_pad * zs + j;
                    for (int c0 = 0; c0 < m_pad; c0 += 32) {
                        uint32_t r[32];
                        tc::tmem_ld32(ctmem + ((uint32_t)(q * 32) << 16) + hh * (uint32_t)m_pad + (uint32_t)c0, r);
                        tc::tmem_ld_wait();
                        float2* zz = z + (int64_t)c0 * zs;
                        if (fb == 0) {
#pragma unroll
                            for (int jj = 0; jj < 32; ++jj) zz[jj * zs] = make_float2(__uint_as_float(r[jj]), 0.f);
                        } else {
#pragma unroll
                            for (int jj = 0; jj < 32; ++jj) {
                                float2 v = zz[jj * zs];
                                df_add(v.x, v.y, __uint_as_float(r[jj]));
                                zz[jj * zs] = v;
                            }
                        }
                    }
                }
                tc::fence_before_sync();
                tc::mbar_arrive(&hd->ctempty);
            }
        }
    }
    // after an abort each MMA thread (producer: warp 1, consumer: warp 7) waits for its MMAs
    if (lane == 0 && *abort_flag) {
        if (warp == 1 && producer) tc::drain_mmas(&hd->pdrain, status);
        if (warp == 7 && consumer) tc::drain_mmas(&hd->cdrain, status);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 512);
    }
}

// ---------------------------------------------------------------- FP32 data: 3xTF32
//
// FP32 X on kind::tf32 tensor cores with FP32-class accuracy: every operand is
// split into a TF32 head (cvt.rna) and the FP32 residual, and the products
// hi*hi + hi*lo + lo*hi are accumulated in FP32 (the lo*lo term is below
// 2^-22 of the result).  Transform warps (6-9) make the X operands in shared
// memory: for Y = X V they round the TMA-loaded tile in place and write the
// residual in the same swizzled layout; for Z = X^T Y they read an unswizzled
// tile and write the transposed head and residual directly in the K-major
// 128-byte-swizzled layout, so no MN-major TF32 operand is needed.
constexpr int kF32Threads = 320;
constexpr int kBK32 = 32;               // K extent of one stage (32 FP32 = 128 B)

struct F32Header {
    uint64_t full[kMaxStages], xform[kMaxStages], empty[kMaxStages];
    uint64_t tfull[2], tempty[2];
    uint64_t drain;                 // the MMA thread's completion barrier after an abort
    uint32_t tmem_base;
    int abort;
};

__device__ inline void f32_prologue(F32Header* hd, int stages, uint32_t tmem_cols, const CUtensorMap* m0,
                                    const CUtensorMap* m1) {
    const int warp = threadIdx.x / 32;
    if (threadIdx.x == 0) {
        for (int i = 0; i < stages; ++i) {
            tc::mbar_init(&hd->full[i], 1);
            tc::mbar_init(&hd->xform[i], 128);           // four transform warps (6-9)
            tc::mbar_init(&hd->empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&hd->tfull[i], 1);
            tc::mbar_init(&hd->tempty[i], 128);
        }
        tc::mbar_init(&hd->drain, 1);
        hd->abort = 0;
        tc::mbar_init_fence();
        tc::tma_prefetch(m0);
        tc::tma_prefetch(m1);
    }
    if (warp == 1) tc::tmem_alloc(&hd->tmem_base, tmem_cols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

// After an abort the MMA thread (warp 1, lane 0) first waits for its MMAs.
__device__ inline void f32_teardown(F32Header* hd, uint32_t tmem_cols, int* status) {
    if (threadIdx.x == 32 && *(volatile int*)&hd->abort) tc::drain_mmas(&hd->drain, status);
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x / 32 == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(hd->tmem_base, tmem_cols);
    }
}

// One 3xTF32 K-stage (32 wide): D += Ahi*Bhi + Ahi*Blo + Alo*Bhi.
__device__ __forceinline__ void mma_3xtf32_stage(uint32_t d_tmem, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi,
                                                 uint32_t b_lo, uint32_t idesc, bool first) {
#pragma unroll
    for (int kk = 0; kk < kBK32 / 8; ++kk) {
        const uint64_t ah = tc::smem_desc_sw128(a_hi + kk * 32, 16, 1024);
        const uint64_t al = tc::smem_desc_sw128(a_lo + kk * 32, 16, 1024);
        const uint64_t bh = tc::smem_desc_sw128(b_hi + kk * 32, 16, 1024);
        const uint64_t bl = tc::smem_desc_sw128(b_lo + kk * 32, 16, 1024);
        tc::mma_tf32(d_tmem, ah, bh, idesc, !(first && kk == 0));
        tc::mma_tf32(d_tmem, ah, bl, idesc, 1);
        tc::mma_tf32(d_tmem, al, bh, idesc, 1);
    }
}

// Y = X V for FP32 X.  Stage: [A head 16 KB][A residual 16 KB][V head][V residual].
// Split K: with ksplit > 1 a task is (tile t, K-range ks) and writes its FP32 partial Y rows to
// Ypart[ks][row][m_pad] (summed and split by ypart_reduce_f32_kernel), so that a minibatch of few
// row tiles still spreads over the SMs.
__global__ void __launch_bounds__(kF32Threads, 1)
    xv_f32_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmV, int ntiles, int nk,
                  int m_pad, int stages, float* __restrict__ Yt, int64_t ldy, int ksplit, float* __restrict__ Ypart,
                  int* status, const int64_t* __restrict__ row0) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* tiles = align1024(smem_raw);
    const uint32_t a_bytes = 128u * 128u;
    const uint32_t b_piece = (uint32_t)m_pad * 128u;
    const uint32_t stage_bytes = 2u * a_bytes + 2u * b_piece;
    F32Header* hd = reinterpret_cast<F32Header*>(tiles + (size_t)stages * stage_bytes);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const uint32_t tmem_cols = tmem_cols_for(m_pad);
    f32_prologue(hd, stages, tmem_cols, &tmX, &tmV);
    const uint32_t tmem = hd->tmem_base;
    volatile int* abort_flag = &hd->abort;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            const int xr0 = row0 ? (int)*row0 : 0;     // device-side first row of X (graph-replayed steps)
            for (int task = blockIdx.x; task < ntiles * ksplit && ok; task += gridDim.x) {
                const int t = task / ksplit, ks = task % ksplit;
                const int k0 = (int)((int64_t)ks * nk / ksplit), k1 = (int)((int64_t)(ks + 1) * nk / ksplit);
                for (int k = k0; k < k1; ++k, ++it) {
                    const uint32_t s = it % stages, ph = (it / stages) & 1u;
                    if (!tc::mbar_wait(&hd->empty[s], ph ^ 1u, status) || *abort_flag) {
                        *abort_flag = 1;
                        ok = false;
                        break;
                    }
                    tc::mbar_expect_tx(&hd->full[s], a_bytes + 2u * b_piece);
                    uint8_t* st = tiles + (size_t)s * stage_bytes;
                    tc::tma_load_2d(st, &tmX, &hd->full[s], k * kBK32, xr0 + t * 128);
                    tc::tma_load_2d(st + 2 * a_bytes, &tmV, &hd->full[s], k * kBK32, 0);
                    tc::tma_load_2d(st + 2 * a_bytes + b_piece, &tmV, &hd->full[s], k * kBK32, m_pad);
                }
            }
            const uint32_t first = it > (uint32_t)stages ? it - (uint32_t)stages : 0u;
            if (*abort_flag)
                for (uint32_t j = first; j < it; ++j)
                    tc::mbar_wait(&hd->full[j % stages], (j / stages) & 1u, status, 100000000ull);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_tf32(128, m_pad);
            uint32_t it = 0, tl = 0;
            bool ok = true;
            for (int task = blockIdx.x; task < ntiles * ksplit && ok; task += gridDim.x, ++tl) {
                const int ks = task % ksplit;
                const int k0 = (int)((int64_t)ks * nk / ksplit), k1 = (int)((int64_t)(ks + 1) * nk / ksplit);
                const uint32_t b = tl & 1u, tph = (tl >> 1) & 1u;
                if (!tc::mbar_wait(&hd->tempty[b], tph ^ 1u, status) || *abort_flag) {
                    *abort_flag = 1;
                    break;
                }
                tc::fence_after_sync();
                for (int k = k0; k < k1; ++k, ++it) {
                    const uint32_t s = it % stages, ph = (it / stages) & 1u;
                    if (!tc::mbar_wait(&hd->xform[s], ph, status) || *abort_flag) {
                        *abort_flag = 1;
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t a = tc::smem_u32(tiles + (size_t)s * stage_bytes);
                    mma_3xtf32_stage(tmem + b * (uint32_t)m_pad, a, a + a_bytes, a + 2 * a_bytes,
                                     a + 2 * a_bytes + b_piece, idesc, k == k0);
                    tc::mma_commit(&hd->empty[s]);
                }
                if (ok) tc::mma_commit(&hd->tfull[b]);
            }
        }
    } else if (warp < 6) {
        const int q = warp & 3;
        uint32_t tl = 0;
        for (int task = blockIdx.x; task < ntiles * ksplit; task += gridDim.x, ++tl) {
            const int t = task / ksplit, ks = task % ksplit;
            const uint32_t b = tl & 1u, tph = (tl >> 1) & 1u;
            if (!tc::mbar_wait(&hd->tfull[b], tph, status) || *abort_flag) {
                *abort_flag = 1;
                break;
            }
            tc::fence_after_sync();
            const int64_t row = (int64_t)t * 128 + q * 32 + lane;
            for (int c0 = 0; c0 < m_pad; c0 += 32) {
                uint32_t r[32];
                tc::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + b * (uint32_t)m_pad + (uint32_t)c0, r);
                tc::tmem_ld_wait();
                if (ksplit == 1) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float y = __uint_as_float(r[j]);
                        const float hi = tc::tf32_rna(y);
                        Yt[(int64_t)(c0 + j) * ldy + row] = hi;
                        Yt[(int64_t)(m_pad + c0 + j) * ldy + row] = y - hi;
                    }
                } else {
                    float4* dst = reinterpret_cast<float4*>(Ypart + ((int64_t)ks * ldy + row) * m_pad + c0);
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        dst[j] = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                                             __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
                }
            }
            tc::fence_before_sync();
            tc::mbar_arrive(&hd->tempty[b]);
        }
    } else {
        // transform: round the X tile to TF32 in place, residual into the next 16 KB
        const int tid = threadIdx.x - 192;
        uint32_t it = 0;
        for (int task = blockIdx.x; task < ntiles * ksplit; task += gridDim.x) {
            const int ks = task % ksplit;
            const int k0 = (int)((int64_t)ks * nk / ksplit), k1 = (int)((int64_t)(ks + 1) * nk / ksplit);
            bool ok = true;
            for (int k = k0; k < k1; ++k, ++it) {
                const uint32_t s = it % stages, ph = (it / stages) & 1u;
                if (!tc::mbar_wait(&hd->full[s], ph, status) || *abort_flag) {
                    *abort_flag = 1;
                    ok = false;
                    break;
                }
                float4* hi = reinterpret_cast<float4*>(tiles + (size_t)s * stage_bytes);
                float4* lo = reinterpret_cast<float4*>(tiles + (size_t)s * stage_bytes + a_bytes);
#pragma unroll
                for (int v = 0; v < 8; ++v) {
                    const int idx = v * 128 + tid;
                    float4 x = hi[idx];
                    float4 h = make_float4(tc::tf32_rna(x.x), tc::tf32_rna(x.y), tc::tf32_rna(x.z), tc::tf32_rna(x.w));
                    hi[idx] = h;
                    lo[idx] = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
                }
                tc::fence_proxy_async_shared();
                tc::mbar_arrive(&hd->xform[s]);
            }
            if (!ok) break;
        }
    }
    f32_teardown(hd, tmem_cols, status);
}

// Z = X^T Y for FP32 X.  Stage: [raw X 4 x (32 x 32) 16 KB][A head 16 KB][A residual 16 KB][Y head][Y residual].
__global__ void __launch_bounds__(kF32Threads, 1)
    xty_f32_kernel(const __grid_constant__ CUtensorMap tmXr, const __grid_constant__ CUtensorMap tmY, int Dt, int Sg,
                   int kst, int flush, int m_pad, int stages, float* __restrict__ Zacc, int* status,
                   const int64_t* __restrict__ row0) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* tiles = align1024(smem_raw);
    const uint32_t a_bytes = 128u * 128u;
    const uint32_t b_piece = (uint32_t)m_pad * 128u;
    const uint32_t stage_bytes = 3u * a_bytes + 2u * b_piece;
    F32Header* hd = reinterpret_cast<F32Header*>(tiles + (size_t)stages * stage_bytes);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const uint32_t tmem_cols = tmem_cols_for(m_pad);
    f32_prologue(hd, stages, tmem_cols, &tmXr, &tmY);
    const uint32_t tmem = hd->tmem_base;
    const int ntask = Dt * Sg;
    volatile int* abort_flag = &hd->abort;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            const int xr0 = row0 ? (int)*row0 : 0;     // device-side first row of X (graph-replayed steps)
            for (int task = blockIdx.x; task < ntask && ok; task += gridDim.x) {
                const int s = task % Dt, g = task / Dt;
                const int k0 = (int)((int64_t)g * kst / Sg), k1 = (int)((int64_t)(g + 1) * kst / Sg);
                for (int k = k0; k < k1; ++k, ++it) {
                    const uint32_t si = it % stages, ph = (it / stages) & 1u;
                    if (!tc::mbar_wait(&hd->empty[si], ph ^ 1u, status) || *abort_flag) {
                        *abort_flag = 1;
                        ok = false;
                        break;
                    }
                    tc::mbar_expect_tx(&hd->full[si], a_bytes + 2u * b_piece);
                    uint8_t* st = tiles + (size_t)si * stage_bytes;
#pragma unroll
                    for (int bx = 0; bx < 4; ++bx)
                        tc::tma_load_2d(st + bx * 4096, &tmXr, &hd->full[si], s * 128 + bx * 32, xr0 + k * kBK32);
                    tc::tma_load_2d(st + 3 * a_bytes, &tmY, &hd->full[si], k * kBK32, 0);
                    tc::tma_load_2d(st + 3 * a_bytes + b_piece, &tmY, &hd->full[si], k * kBK32, m_pad);
                }
            }
            const uint32_t first = it > (uint32_t)stages ? it - (uint32_t)stages : 0u;
            if (*abort_flag)
                for (uint32_t j = first; j < it; ++j)
                    tc::mbar_wait(&hd->full[j % stages], (j / stages) & 1u, status, 100000000ull);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_tf32(128, m_pad);
            uint32_t it = 0, fb = 0;
            bool ok = true;
            for (int task = blockIdx.x; task < ntask && ok; task += gridDim.x) {
                const int g = task / Dt;
                const int k0 = (int)((int64_t)g * kst / Sg), k1 = (int)((int64_t)(g + 1) * kst / Sg);
                for (int kb = k0; kb < k1 && ok; kb += flush, ++fb) {
                    const int ke = kb + flush < k1 ? kb + flush : k1;
                    const uint32_t b = fb & 1u, tph = (fb >> 1) & 1u;
                    if (!tc::mbar_wait(&hd->tempty[b], tph ^ 1u, status) || *abort_flag) {
                        *abort_flag = 1;
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    for (int k = kb; k < ke; ++k, ++it) {
                        const uint32_t si = it % stages, ph = (it / stages) & 1u;
                        if (!tc::mbar_wait(&hd->xform[si], ph, status) || *abort_flag) {
                            *abort_flag = 1;
                            ok = false;
                            break;
                        }
                        tc::fence_after_sync();
                        const uint32_t a = tc::smem_u32(tiles + (size_t)si * stage_bytes);
                        mma_3xtf32_stage(tmem + b * (uint32_t)m_pad, a + a_bytes, a + 2 * a_bytes, a + 3 * a_bytes,
                                         a + 3 * a_bytes + b_piece, idesc, k == kb);
                        tc::mma_commit(&hd->empty[si]);
                    }
                    if (ok) tc::mma_commit(&hd->tfull[b]);
                }
            }
        }
    } else if (warp < 6) {
        const int q = warp & 3;
        uint32_t fb = 0;
        bool ok = true;
        for (int task = blockIdx.x; task < ntask && ok; task += gridDim.x) {
            const int s = task % Dt, g = task / Dt;
            const int k0 = (int)((int64_t)g * kst / Sg), k1 = (int)((int64_t)(g + 1) * kst / Sg);
            const int64_t j = (int64_t)s * 128 + q * 32 + lane;
            const int64_t zs = (int64_t)Dt * 128;     // Z partials [g][column][row]: a warp's rows contiguous
            float2* z = reinterpret_cast<float2*>(Zacc) + (int64_t)g * m_pad * zs + j;
            for (int kb = k0; kb < k1; kb += flush, ++fb) {
                const uint32_t b = fb & 1u, tph = (fb >> 1) & 1u;
                if (!tc::mbar_wait(&hd->tfull[b], tph, status) || *abort_flag) {
                    *abort_flag = 1;
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                for (int c0 = 0; c0 < m_pad; c0 += 32) {
                    uint32_t r[32];
                    tc::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + b * (uint32_t)m_pad + (uint32_t)c0, r);
                    tc::tmem_ld_wait();
                    float2* zz = z + (int64_t)c0 * zs;
                    if (kb == k0) {
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj) zz[jj * zs] = make_float2(__uint_as_float(r[jj]), 0.f);
                    } else {
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj) {
                            float2 v = zz[jj * zs];
                            df_add(v.x, v.y, __uint_as_float(r[jj]));
                            zz[jj * zs] = v;
                        }
                    }
                }
                tc::fence_before_sync();
                tc::mbar_arrive(&hd->tempty[b]);
            }
        }
    } else {
        // transform: column i of the 128-column slice -> row i of the K-major
        // operands (head and residual), 128-byte swizzle: 16-byte chunk c of row
        // i is stored at chunk position c ^ (i % 8) of its 1024-byte atom.
        const int i = threadIdx.x - 192;
        const float* raw_col = nullptr;
        uint32_t it = 0;
        bool ok = true;
        for (int task = blockIdx.x; task < ntask && ok; task += gridDim.x) {
            const int g = task / Dt;
            const int k0 = (int)((int64_t)g * kst / Sg), k1 = (int)((int64_t)(g + 1) * kst / Sg);
            for (int k = k0; k < k1; ++k, ++it) {
                const uint32_t si = it % stages, ph = (it / stages) & 1u;
                if (!tc::mbar_wait(&hd->full[si], ph, status) || *abort_flag) {
                    *abort_flag = 1;
                    ok = false;
                    break;
                }
                uint8_t* st = tiles + (size_t)si * stage_bytes;
                raw_col = reinterpret_cast<const float*>(st + (i / 32) * 4096) + (i % 32);
                uint8_t* hi_row = st + a_bytes + (i / 8) * 1024 + (i % 8) * 128;
                uint8_t* lo_row = st + 2 * a_bytes + (i / 8) * 1024 + (i % 8) * 128;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    float x[4], h[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        x[e] = raw_col[(c * 4 + e) * 32];
                        h[e] = tc::tf32_rna(x[e]);
                    }
                    const int pos = (c ^ (i % 8)) * 16;
                    *reinterpret_cast<float4*>(hi_row + pos) = make_float4(h[0], h[1], h[2], h[3]);
                    *reinterpret_cast<float4*>(lo_row + pos) =
                        make_float4(x[0] - h[0], x[1] - h[1], x[2] - h[2], x[3] - h[3]);
                }
                tc::fence_proxy_async_shared();
                tc::mbar_arrive(&hd->xform[si]);
            }
        }
    }
    f32_teardown(hd, tmem_cols, status);
}

// V (d x m column-major FP32) -> TF32 head and FP32 residual, [2][m_pad][ldv4], zero padded.
__global__ void split_v_f32_kernel(const float* __restrict__ V, int64_t d, int m, int m_pad, int64_t ldv4,
                                   float* __restrict__ Vp) {
    const int64_t total = (int64_t)m_pad * ldv4;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / ldv4);
        const int64_t j = e % ldv4;
        const float v = (c < m && j < d) ? V[(int64_t)c * d + j] : 0.f;
        const float h = tc::tf32_rna(v);
        Vp[e] = h;
        Vp[e + total] = v - h;
    }
}

// V (d x m column-major FP32) -> S BF16 pieces, [S][m_pad][ldv], zero padded.
template <int S>
__global__ void split_v_kernel(const float* __restrict__ V, int64_t d, int m, int m_pad, int64_t ldv,
                               __nv_bfloat16* __restrict__ Vp) {
    const int64_t total = (int64_t)m_pad * ldv;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / ldv);
        const int64_t j = e % ldv;
        const float v = (c < m && j < d) ? V[(int64_t)c * d + j] : 0.f;
        split_store<S>(v, Vp + e, total);
    }
}

// Y = sum over the K-ranges of the split-K partials, then the S BF16 pieces of Y^T.
template <int S>
__global__ void ypart_reduce_kernel(const float* __restrict__ Ypart, int ksplit, int64_t ldy, int m_pad,
                                    __nv_bfloat16* __restrict__ Yt) {
    const int64_t total = ldy * m_pad;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = e / m_pad;
        const int c = (int)(e % m_pad);
        float acc = 0.f;
        for (int ks = 0; ks < ksplit; ++ks) acc += Ypart[(int64_t)ks * total + e];
        split_store<S>(acc, Yt + (int64_t)c * ldy + row, (int64_t)m_pad * ldy);
    }
}

// FP32 data: Y = sum over the K-ranges of the split-K partials, then its TF32 head and FP32 residual.
__global__ void ypart_reduce_f32_kernel(const float* __restrict__ Ypart, int ksplit, int64_t ldy, int m_pad,
                                        float* __restrict__ Yt) {
    const int64_t total = ldy * m_pad;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = e / m_pad;
        const int c = (int)(e % m_pad);
        float acc = 0.f;
        for (int ks = 0; ks < ksplit; ++ks) acc += Ypart[(int64_t)ks * total + e];
        const float hi = tc::tf32_rna(acc);
        Yt[(int64_t)c * ldy + row] = hi;
        Yt[(int64_t)(m_pad + c) * ldy + row] = acc - hi;
    }
}

__global__ void zreduce_kernel(const float* __restrict__ Zacc, int Sg, int Dt, int64_t d, int m, int m_pad,
                               float* __restrict__ Z) {
    const int64_t total = d * m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / d);
        const int64_t j = e % d;
        float hi = 0.f, lo = 0.f;
        for (int g = 0; g < Sg; ++g) {
            const float2 v = reinterpret_cast<const float2*>(Zacc)[((int64_t)g * m_pad + c) * (Dt * 128) + j];
            df_add(hi, lo, v.x);
            df_add(hi, lo, v.y);
        }
        Z[e] = hi + lo;
    }
}

// ---------------------------------------------------------------- grouped fast BF16 pass
//
// The two-kernel fast pass of many instances in one launch each (grouped.h).
// A Z item's K range (a row group) is at most 128 K-stages, inside the fold
// interval, so each item leaves one FP32 partial, summed in double-float by
// zreduce_grouped_kernel.
// work item w of Y = X V is tile w - base[i] of instance i, of Z = X^T Y task
// w - base[i] (128-column slice s, row group g) of instance i.  Each item uses
// its instance's TMA descriptors (device memory), basis width (the MMA's N)
// and buffers; the shared-memory stages and TMEM are sized for the widest basis.

__global__ void split_q_grouped_kernel(const GInst* __restrict__ gi, GTable tab) {
    const int i = group_find(tab, blockIdx.x);
    const GInst& g = gi[i];
    const int64_t total = (int64_t)g.m_pad * g.ldv;
    const int64_t e = (int64_t)(blockIdx.x - tab.base[i]) * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int c = (int)(e / g.ldv);
    const int64_t k = e % g.ldv;
    const float v = (c < g.m && k < g.d) ? g.Z[(int64_t)c * g.d + k] : 0.f;
    split_store<3>(v, g.Q3 + e, total);
}

__global__ void zreduce_grouped_kernel(const GInst* __restrict__ gi, GTable tab) {
    const int i = group_find(tab, blockIdx.x);
    const GInst& g = gi[i];
    // an instance's d m (< 2^31) fits 32-bit index arithmetic
    const int e = (blockIdx.x - tab.base[i]) * blockDim.x + threadIdx.x;
    const int d = (int)g.d;
    if (e >= d * g.m) return;
    const int c = e / d, j = e - c * d;
    const int64_t stride = (int64_t)g.m_pad * (g.Dt * 128);
    const float* p = g.Zacc + (int64_t)c * (g.Dt * 128) + j;
    float hi = 0.f, lo = 0.f;
    for (int q = 0; q < g.Sg; ++q) df_add(hi, lo, p[q * stride]);
    g.Z[e] = hi + lo;
}

__global__ void __launch_bounds__(kThreads, 1)
    xv_grouped_kernel(const GInst* __restrict__ gi, const GMaps* __restrict__ maps, GTable items, int stages,
                      int* status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* tiles = align1024(smem_raw);
    const uint32_t a_bytes = 128u * 128u, b_max = 128u * 128u;
    const uint32_t stage_bytes = a_bytes + b_max;
    SmemHeader* hd = reinterpret_cast<SmemHeader*>(tiles + (size_t)stages * stage_bytes);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const uint32_t tmem_cols = 256;
    tc_prologue(hd, stages, tmem_cols, &maps[0].xa, &maps[0].v);
    const uint32_t tmem = hd->tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            for (int w = blockIdx.x; w < items.total && ok; w += gridDim.x) {
                const int i = group_find(items, w), t = w - items.base[i];
                const GInst& g = gi[i];
                const uint32_t bytes = a_bytes + (uint32_t)g.m_pad * 128u;
                for (int k = 0; k < g.nk; ++k, ++it) {
                    const uint32_t s = it % stages, ph = (it / stages) & 1u;
                    if (!tc::mbar_wait(&hd->empty[s], ph ^ 1u, status) || *(volatile int*)&hd->abort) {
                        hd->abort = 1;
                        ok = false;
                        break;
                    }
                    tc::mbar_expect_tx(&hd->full[s], bytes);
                    uint8_t* st = tiles + (size_t)s * stage_bytes;
                    tc::tma_load_2d(st, &maps[i].xa, &hd->full[s], k * kBK, t * 128);
                    tc::tma_load_2d(st + a_bytes, &maps[i].v, &hd->full[s], k * kBK, 0);
                }
            }
            if (!ok) drain_copies(hd, it, stages, status);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            uint32_t it = 0, tl = 0;
            bool ok = true;
            for (int w = blockIdx.x; w < items.total && ok; w += gridDim.x, ++tl) {
                const GInst& g = gi[group_find(items, w)];
                const uint32_t idesc = tc::idesc_bf16(128, g.m_pad, false, false);
                const uint32_t b = tl & 1u, tph = (tl >> 1) & 1u;
                if (!tc::mbar_wait(&hd->tempty[b], tph ^ 1u, status) || *(volatile int*)&hd->abort) {
                    hd->abort = 1;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t d_tmem = tmem + b * 128u;
                for (int k = 0; k < g.nk; ++k, ++it) {
                    const uint32_t s = it % stages, ph = (it / stages) & 1u;
                    if (!tc::mbar_wait(&hd->full[s], ph, status) || *(volatile int*)&hd->abort) {
                        hd->abort = 1;
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t a_addr = tc::smem_u32(tiles + (size_t)s * stage_bytes);
#pragma unroll
                    for (int kk = 0; kk < kBK / 16; ++kk) {
                        const uint64_t adesc = tc::smem_desc_sw128(a_addr + kk * 32, 16, 1024);
                        const uint64_t bdesc = tc::smem_desc_sw128(a_addr + a_bytes + kk * 32, 16, 1024);
                        tc::mma_f16(d_tmem, adesc, bdesc, idesc, (k != 0 || kk != 0) ? 1u : 0u);
                    }
                    tc::mma_commit(&hd->empty[s]);
                }
                if (ok) tc::mma_commit(&hd->tfull[b]);
            }
        }
    } else {
        const int q = warp & 3;
        uint32_t tl = 0;
        for (int w = blockIdx.x; w < items.total; w += gridDim.x, ++tl) {
            const int i = group_find(items, w), t = w - items.base[i];
            const GInst& g = gi[i];
            const uint32_t b = tl & 1u, tph = (tl >> 1) & 1u;
            if (!tc::mbar_wait(&hd->tfull[b], tph, status) || *(volatile int*)&hd->abort) {
                hd->abort = 1;
                break;
            }
            tc::fence_after_sync();
            const int64_t row = (int64_t)t * 128 + q * 32 + lane;
            for (int c0 = 0; c0 < g.m_pad; c0 += 32) {
                uint32_t r[32];
                tc::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + b * 128u + (uint32_t)c0, r);
                tc::tmem_ld_wait();
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    g.Yt[(int64_t)(c0 + j) * g.ldy + row] = __float2bfloat16_rn(__uint_as_float(r[j]));
            }
            tc::fence_before_sync();
            tc::mbar_arrive(&hd->tempty[b]);
        }
    }
    tc_epilogue_teardown(hd, tmem_cols, status);
}

__global__ void __launch_bounds__(kThreads, 1)
    xty_grouped_kernel(const GInst* __restrict__ gi, const GMaps* __restrict__ maps, GTable items, int flush,
                       int stages, int* status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* tiles = align1024(smem_raw);
    const uint32_t a_bytes = 2u * 64u * 128u, b_max = 128u * 128u;
    const uint32_t stage_bytes = a_bytes + b_max;
    SmemHeader* hd = reinterpret_cast<SmemHeader*>(tiles + (size_t)stages * stage_bytes);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const uint32_t tmem_cols = 256;
    tc_prologue(hd, stages, tmem_cols, &maps[0].xb, &maps[0].y);
    const uint32_t tmem = hd->tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            for (int w = blockIdx.x; w < items.total && ok; w += gridDim.x) {
                const int i = group_find(items, w), task = w - items.base[i];
                const GInst& g = gi[i];
                const int s = task % g.Dt, grp = task / g.Dt;
                const int k0 = (int)((int64_t)grp * g.kst / g.Sg), k1 = (int)((int64_t)(grp + 1) * g.kst / g.Sg);
                const uint32_t bytes = a_bytes + (uint32_t)g.m_pad * 128u;
                for (int k = k0; k < k1; ++k, ++it) {
                    const uint32_t st_i = it % stages, ph = (it / stages) & 1u;
                    if (!tc::mbar_wait(&hd->empty[st_i], ph ^ 1u, status) || *(volatile int*)&hd->abort) {
                        hd->abort = 1;
                        ok = false;
                        break;
                    }
                    tc::mbar_expect_tx(&hd->full[st_i], bytes);
                    uint8_t* st = tiles + (size_t)st_i * stage_bytes;
                    tc::tma_load_2d(st, &maps[i].xb, &hd->full[st_i], s * 128, k * kBK);
                    tc::tma_load_2d(st + 8192, &maps[i].xb, &hd->full[st_i], s * 128 + 64, k * kBK);
                    tc::tma_load_2d(st + a_bytes, &maps[i].y, &hd->full[st_i], k * kBK, 0);
                }
            }
            if (!ok) drain_copies(hd, it, stages, status);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            uint32_t it = 0, fb = 0;
            bool ok = true;
            for (int w = blockIdx.x; w < items.total && ok; w += gridDim.x) {
                const int i = group_find(items, w), task = w - items.base[i];
                const GInst& g = gi[i];
                const uint32_t idesc = tc::idesc_bf16(128, g.m_pad, true, false);
                const int grp = task / g.Dt;
                const int k0 = (int)((int64_t)grp * g.kst / g.Sg), k1 = (int)((int64_t)(grp + 1) * g.kst / g.Sg);
                for (int kb = k0; kb < k1 && ok; kb += flush, ++fb) {
                    const int ke = kb + flush < k1 ? kb + flush : k1;
                    const uint32_t b = fb & 1u, tph = (fb >> 1) & 1u;
                    if (!tc::mbar_wait(&hd->tempty[b], tph ^ 1u, status) || *(volatile int*)&hd->abort) {
                        hd->abort = 1;
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t d_tmem = tmem + b * 128u;
                    for (int k = kb; k < ke; ++k, ++it) {
                        const uint32_t st_i = it % stages, ph = (it / stages) & 1u;
                        if (!tc::mbar_wait(&hd->full[st_i], ph, status) || *(volatile int*)&hd->abort) {
                            hd->abort = 1;
                            ok = false;
                            break;
                        }
                        tc::fence_after_sync();
                        const uint32_t a_addr = tc::smem_u32(tiles + (size_t)st_i * stage_bytes);
#pragma unroll
                        for (int kk = 0; kk < kBK / 16; ++kk) {
                            const uint64_t adesc = tc::smem_desc_sw128(a_addr + kk * 2048, 8192, 1024);
                            const uint64_t bdesc = tc::smem_desc_sw128(a_addr + a_bytes + kk * 32, 16, 1024);
                            tc::mma_f16(d_tmem, adesc, bdesc, idesc, (k != kb) || kk != 0);
                        }
                        tc::mma_commit(&hd->empty[st_i]);
                    }
                    if (ok) tc::mma_commit(&hd->tfull[b]);
                }
            }
        }
    } else {
        const int q = warp & 3;
        uint32_t fb = 0;
        bool ok = true;
        for (int w = blockIdx.x; w < items.total && ok; w += gridDim.x) {
            const int i = group_find(items, w), task = w - items.base[i];
            const GInst& g = gi[i];
            const int s = task % g.Dt, grp = task / g.Dt;
            const int k0 = (int)((int64_t)grp * g.kst / g.Sg), k1 = (int)((int64_t)(grp + 1) * g.kst / g.Sg);
            const int64_t j = (int64_t)s * 128 + q * 32 + lane;
            const int64_t zs = (int64_t)g.Dt * 128;     // Z partials [g][column][row], FP32
            float* z = g.Zacc + (int64_t)grp * g.m_pad * zs + j;
            for (int kb = k0; kb < k1; kb += flush, ++fb) {
                const uint32_t b = fb & 1u, tph = (fb >> 1) & 1u;
                if (!tc::mbar_wait(&hd->tfull[b], tph, status) || *(volatile int*)&hd->abort) {
                    hd->abort = 1;
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                for (int c0 = 0; c0 < g.m_pad; c0 += 32) {
                    uint32_t r[32];
                    tc::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + b * 128u + (uint32_t)c0, r);
                    tc::tmem_ld_wait();
                    // one fold per item (its K range is at most `flush` stages): store
#pragma unroll
                    for (int jj = 0; jj < 32; ++jj) z[(int64_t)(c0 + jj) * zs] = __uint_as_float(r[jj]);
                }
                tc::fence_before_sync();
                tc::mbar_arrive(&hd->tempty[b]);
            }
        }
    }
    tc_epilogue_teardown(hd, tmem_cols, status);
}

// ---------------------------------------------------------------- host side

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

bool encode_2d(CUtensorMap* map, CUtensorMapDataType dt, const void* base, uint64_t inner, uint64_t outer,
               uint64_t pitch_bytes, uint32_t box_inner, uint32_t box_outer, CUtensorMapSwizzle swz) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {pitch_bytes};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool encode_bf16_2d(CUtensorMap* map, const void* base, uint64_t inner, uint64_t outer, uint64_t pitch_bytes,
                    uint32_t box_inner, uint32_t box_outer) {
    return encode_2d(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, base, inner, outer, pitch_bytes, box_inner, box_outer,
                     CU_TENSOR_MAP_SWIZZLE_128B);
}

cudaError_t launch_split_v(const float* V, int64_t d, int m, int m_pad, int64_t ldv, int S, __nv_bfloat16* Vp,
                           cudaStream_t st) {
    const int64_t total = (int64_t)m_pad * ldv;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    note_launch();
    if (S == 1)
        split_v_kernel<1><<<blocks, 256, 0, st>>>(V, d, m, m_pad, ldv, Vp);
    else if (S == 2)
        split_v_kernel<2><<<blocks, 256, 0, st>>>(V, d, m, m_pad, ldv, Vp);
    else
        split_v_kernel<3><<<blocks, 256, 0, st>>>(V, d, m, m_pad, ldv, Vp);
    return cudaGetLastError();
}

namespace {

int stages_for(uint32_t stage_bytes) {
    int s = (int)((kSmemBudget - 2048) / stage_bytes);
    return s < 2 ? 2 : (s > kMaxStages ? kMaxStages : s);
}

size_t smem_bytes(int stages, uint32_t stage_bytes) { return 1024 + (size_t)stages * stage_bytes + sizeof(SmemHeader); }

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }
inline int m_pad_of(int m) { return (int)round_up(m, 32); }

struct Layout {
    int64_t ldv, ldy, rows_pad_max;
    int m_pad, Dt;
    size_t vp_bytes, yt_bytes, z_bytes, flag_bytes;
};

Layout layout_of(int64_t n, int64_t d, int m, int num_sms) {
    Layout L;
    L.m_pad = 128;                                   // scratch sized for the largest m
    L.ldv = round_up(d, 8);
    L.rows_pad_max = round_up(n, 128);
    L.Dt = (int)((d + 127) / 128);
    // sized for the larger of three BF16 pieces and two FP32 pieces
    L.vp_bytes = std::max((size_t)3 * L.m_pad * L.ldv * 2, (size_t)2 * L.m_pad * round_up(d, 4) * 4);
    L.yt_bytes = std::max((size_t)3 * L.m_pad * L.rows_pad_max * 2, (size_t)2 * L.m_pad * L.rows_pad_max * 4);
    L.z_bytes = (size_t)(2 * num_sms + L.Dt + 2) * 128 * L.m_pad * 8;
    L.flag_bytes = (size_t)10 * (L.rows_pad_max / 128 + 1) * sizeof(int);   // fused pass: 2 + 2 x 4 per tile
    (void)m;
    return L;
}

struct PassShape {
    int64_t d, rows, ldv, ldy;
    int m_pad, Dt, ntiles, nk;
};

// row0_dev (device, may be NULL): the batch's first row, read by the kernels;
// the X descriptors then cover all n rows and r0 only fixes the batch size.
template <int S, bool FP8X = false>
cudaError_t prepare_pass(const XView& x, const float* V, int m, int64_t r0, int64_t r1, const TcPassScratch& sc,
                         PassShape& ps, CUtensorMap& tmXa, CUtensorMap& tmXb, CUtensorMap& tmV, CUtensorMap& tmY,
                         cudaStream_t st, const int64_t* row0_dev = nullptr) {
    ps.d = x.d;
    ps.rows = r1 - r0;
    ps.m_pad = m_pad_of(m);
    ps.ldv = round_up(ps.d, 8);
    ps.ldy = round_up(ps.rows, 128);
    ps.Dt = (int)((ps.d + 127) / 128);
    ps.ntiles = (int)(ps.ldy / 128);
    ps.nk = (int)((ps.d + kBK - 1) / kBK);
    __nv_bfloat16* Vp = static_cast<__nv_bfloat16*>(sc.vp);
    __nv_bfloat16* Yt = static_cast<__nv_bfloat16*>(sc.yt);
    {
        const int64_t total = (int64_t)ps.m_pad * ps.ldv;
        int blocks = (int)((total + 255) / 256);
        if (blocks > 4096) blocks = 4096;
        note_launch();
        split_v_kernel<S><<<blocks, 256, 0, st>>>(V, ps.d, m, ps.m_pad, ps.ldv, Vp);
    }
    const int esz = FP8X ? 1 : 2;
    const void* xbase = static_cast<const char*>(x.ptr) + (row0_dev ? 0 : r0) * x.ld * esz;
    const uint64_t xrows = row0_dev ? (uint64_t)x.n : (uint64_t)ps.rows;
    const bool xmaps = FP8X ? encode_2d(&tmXa, CU_TENSOR_MAP_DATA_TYPE_UINT8, xbase, ps.d, xrows, x.ld, 64, 128,
                                        CU_TENSOR_MAP_SWIZZLE_NONE) &&
                                  encode_2d(&tmXb, CU_TENSOR_MAP_DATA_TYPE_UINT8, xbase, ps.d, xrows, x.ld, 128, 64,
                                            CU_TENSOR_MAP_SWIZZLE_NONE)
                            : encode_bf16_2d(&tmXa, xbase, ps.d, xrows, x.ld * 2, 64, 128) &&
                                  encode_bf16_2d(&tmXb, xbase, ps.d, xrows, x.ld * 2, 64, 64);
    if (!xmaps ||
        !encode_bf16_2d(&tmV, Vp, ps.d, (uint64_t)S * ps.m_pad, ps.ldv * 2, 64, ps.m_pad) ||
        !encode_bf16_2d(&tmY, Yt, ps.ldy, (uint64_t)S * ps.m_pad, ps.ldy * 2, 64, ps.m_pad))
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// Row groups of the Z = X^T Y kernels, whose tasks are (128-column slice, row
// group) and whose CTAs each run whole tasks: Sg minimises a CTA's share,
// ceil(Dt Sg / num_sms) / Sg, within kst (a K-stage per group at least) and the
// capacity of the double-float partials (Dt * 128 * m_pad float2 per group);
// the smallest such Sg.  (Dt = 32 on 152 SMs: 9 groups, 2 tasks per CTA, not 4
// groups on 128 CTAs.)
int choose_row_groups(int Dt, int kst, int num_sms, size_t z_bytes, int m_pad) {
    const size_t per_group = (size_t)Dt * 128 * (size_t)m_pad * 8;
    int cap = (int)std::min<size_t>(z_bytes / per_group, (size_t)std::max(kst, 1));
    if (cap < 1) cap = 1;
    int best = 1;
    double best_cost = 1e300;
    for (int sg = 1; sg <= cap && sg <= 4 * num_sms; ++sg) {
        const int64_t ntask = (int64_t)Dt * sg;
        const double cost = (double)((ntask + num_sms - 1) / num_sms) / sg;
        if (cost < best_cost * (1.0 - 1e-9)) {
            best_cost = cost;
            best = sg;
        }
    }
    return best;
}

cudaError_t launch_zreduce(const float* Zacc, int Sg, int Dt, int64_t d, int m, int m_pad, float* Z, cudaStream_t st) {
    const int64_t total = d * m;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 8192) blocks = 8192;
    note_launch();
    zreduce_kernel<<<blocks, 256, 0, st>>>(Zacc, Sg, Dt, d, m, m_pad, Z);
    return cudaGetLastError();
}

// Two GEMM kernels: Y = X V, then Z = X^T Y (X is read twice).
template <int S, bool FP8X = false>
cudaError_t run_pass(const XView& x, const float* V, int m, int64_t r0, int64_t r1, float* Z, int flush,
                     const TcPassScratch& sc, int* status, int num_sms, cudaStream_t st,
                     const int64_t* row0_dev = nullptr) {
    PassShape ps;
    CUtensorMap tmXa, tmXb, tmV, tmY;
    cudaError_t e = prepare_pass<S, FP8X>(x, V, m, r0, r1, sc, ps, tmXa, tmXb, tmV, tmY, st, row0_dev);
    constexpr int threads = FP8X ? kThreadsFp8 : kThreads;
    constexpr uint32_t raw_xv = FP8X ? 128u * 64u : 0u, raw_xty = FP8X ? 64u * 128u : 0u;
    if (e != cudaSuccess) return e;
    __nv_bfloat16* Yt = static_cast<__nv_bfloat16*>(sc.yt);
    float* Zacc = static_cast<float*>(sc.zacc);
    {
        const uint32_t stage_bytes = raw_xv + 128u * 128u + S * (uint32_t)ps.m_pad * 128u;
        const int stages = stages_for(stage_bytes);
        const size_t smem = smem_bytes(stages, stage_bytes);
        e = smem_at_least(reinterpret_cast<const void*>(xv_tc_kernel<S, FP8X>), smem);
        if (e != cudaSuccess) return e;
        // few row tiles (a minibatch) and a long K: split K so that every SM has work
        int ksplit = 1;
        if (ps.ntiles * 2 <= num_sms && ps.nk >= 8) {
            ksplit = (2 * num_sms + ps.ntiles - 1) / ps.ntiles;
            ksplit = std::min(ksplit, ps.nk / 4);
            const int64_t cap = (int64_t)(sc.z_bytes / ((size_t)ps.ldy * ps.m_pad * sizeof(float)));
            ksplit = (int)std::min<int64_t>(ksplit, cap);
            if (ksplit < 2) ksplit = 1;
        }
        const int ntask = ps.ntiles * ksplit;
        const int grid = ntask < num_sms ? ntask : num_sms;
        float* Ypart = static_cast<float*>(sc.zacc);
        note_launch();
        const float* scales = FP8X ? x.scales + r0 : nullptr;
        xv_tc_kernel<S, FP8X><<<grid, threads, smem, st>>>(tmXa, tmV, ps.ntiles, ps.nk, ps.m_pad, stages, Yt,
                                                            ps.ldy, ksplit, Ypart, scales, ps.rows, status, row0_dev);
        if (ksplit > 1) {
            const int64_t total = ps.ldy * ps.m_pad;
            int blocks = (int)((total + 255) / 256);
            if (blocks > 4096) blocks = 4096;
            note_launch();
            ypart_reduce_kernel<S><<<blocks, 256, 0, st>>>(Ypart, ksplit, ps.ldy, ps.m_pad, Yt);
        }
    }
    int Sg;
    {
        const uint32_t stage_bytes = raw_xty + 2u * 64u * 128u + S * (uint32_t)ps.m_pad * 128u;
        const int stages = stages_for(stage_bytes);
        const size_t smem = smem_bytes(stages, stage_bytes);
        e = smem_at_least(reinterpret_cast<const void*>(xty_tc_kernel<S, FP8X>), smem);
        if (e != cudaSuccess) return e;
        const int kst = (int)(ps.ldy / kBK);
        Sg = choose_row_groups(ps.Dt, kst, num_sms, sc.z_bytes, ps.m_pad);
        const int ntask = ps.Dt * Sg;
        const int grid = ntask < num_sms ? ntask : num_sms;
        note_launch();
        xty_tc_kernel<S, FP8X><<<grid, threads, smem, st>>>(tmXb, tmY, ps.Dt, Sg, kst, flush, ps.m_pad, stages,
                                                              Zacc, status, row0_dev);
    }
    return launch_zreduce(Zacc, Sg, ps.Dt, ps.d, m, ps.m_pad, Z, st);
}

// FAST pass of E4M3 data on the FP8 tensor cores (two kernels, X8 read twice): see xv_f8_kernel.
cudaError_t run_pass_f8(const XView& x, const float* V, int m, int64_t r0, int64_t r1, float* Z, int flush,
                        const TcPassScratch& sc, int* status, int num_sms, cudaStream_t st) {
    const int64_t d = x.d, rows = r1 - r0;
    const int m_pad = m_pad_of(m);
    const int64_t ldv8 = round_up(d, 16), ldy = round_up(rows, 256);
    const int Dt2 = (int)((d + 255) / 256), ntiles = (int)(ldy / 256), nk = (int)((d + 127) / 128);
    uint8_t* V8 = static_cast<uint8_t*>(sc.vp);
    uint8_t* Y8 = static_cast<uint8_t*>(sc.yt);
    float* f8s = reinterpret_cast<float*>(sc.flags);
    float* Zacc = static_cast<float*>(sc.zacc);
    const float* scales = x.scales + r0;
    cudaError_t e = cudaMemsetAsync(f8s, 0, 5 * sizeof(float), st);
    if (e != cudaSuccess) return e;
    note_launch();
    f8_stats_kernel<<<m + 64, 256, 0, st>>>(V, d, m, scales, rows, f8s);
    {
        const int64_t pairs = (int64_t)m_pad * ldv8 / 2;
        int blocks = (int)((pairs + 255) / 256);
        if (blocks > 4096) blocks = 4096;
        note_launch();
        split_v8_kernel<<<blocks, 256, 0, st>>>(V, d, m, m_pad, ldv8, f8s, V8);
    }
    CUtensorMap tmX, tmV, tmY;
    const void* xbase = static_cast<const uint8_t*>(x.ptr) + r0 * x.ld;
    if (!encode_2d(&tmX, CU_TENSOR_MAP_DATA_TYPE_UINT8, xbase, d, rows, x.ld, 128, 128, CU_TENSOR_MAP_SWIZZLE_128B) ||
        !encode_2d(&tmV, CU_TENSOR_MAP_DATA_TYPE_UINT8, V8, ldv8, 2 * (uint64_t)m_pad, ldv8, 128, m_pad,
                   CU_TENSOR_MAP_SWIZZLE_128B) ||
        !encode_2d(&tmY, CU_TENSOR_MAP_DATA_TYPE_UINT8, Y8, ldy, 2 * (uint64_t)m_pad, ldy, 128, m_pad,
                   CU_TENSOR_MAP_SWIZZLE_128B))
        return cudaErrorInvalidValue;
    const uint32_t stage_bytes = 2u * 128u * 128u + 2u * (uint32_t)m_pad * 128u;
    const int stages = stages_for(stage_bytes);
    const size_t smem = smem_bytes(stages, stage_bytes);
    e = smem_at_least(reinterpret_cast<const void*>(xv_f8_kernel), smem);
    if (e != cudaSuccess) return e;
    e = smem_at_least(reinterpret_cast<const void*>(xty_f8_kernel), smem);
    if (e != cudaSuccess) return e;
    note_launch();
    xv_f8_kernel<<<ntiles < num_sms ? ntiles : num_sms, kThreads, smem, st>>>(tmX, tmV, ntiles, nk, m_pad, stages,
                                                                              Y8, ldy, scales, rows, f8s, status);
    const int kst = (int)(ldy / 128);
    // tasks are 256-column slices; a row group's partials hold 2 Dt2 128-column slices
    const int Sg2 = choose_row_groups(Dt2, kst, num_sms, sc.z_bytes / 2, m_pad);
    const int ntask = Dt2 * Sg2;
    note_launch();
    xty_f8_kernel<<<ntask < num_sms ? ntask : num_sms, kThreads, smem, st>>>(tmX, tmY, Dt2, Sg2, kst, flush, m_pad,
                                                                             stages, Zacc, f8s, status);
    return launch_zreduce(Zacc, Sg2, 2 * Dt2, d, m, m_pad, Z, st);
}

// Fused single-read pass (one piece, BF16): see xpass_fused_kernel.
cudaError_t run_fused(const XView& x, const float* V, int m, int64_t r0, int64_t r1, float* Z,
                      const TcPassScratch& sc, const TcSchedule& sched, int* status, int num_sms, cudaStream_t st) {
    PassShape ps;
    CUtensorMap tmXa, tmXb, tmV, tmY;
    cudaError_t e = prepare_pass<1>(x, V, m, r0, r1, sc, ps, tmXa, tmXb, tmV, tmY, st);
    if (e != cudaSuccess) return e;
    const int Dt2 = (ps.Dt + 1) / 2;
    int Sg = num_sms / Dt2;
    if (Sg > ps.ntiles) Sg = ps.ntiles;
    // whole-K tiles unless asked for two K halves (which need at least two K-stages)
    const int kparts = (sched.kparts == 2 && ps.nk >= 2) ? 2 : 1;
    int NP = sched.producers > 0 ? sched.producers : num_sms;
    if (NP > num_sms) NP = num_sms;
    if (NP > ps.ntiles * kparts) NP = ps.ntiles * kparts;
    int window = sched.window > 0 ? sched.window : (NP + kparts - 1) / kparts + 4 * Sg;
    // Share of each tile's K-stages loaded evict_last (the rest evict_first):
    // sched.l2_keep percent, by default what keeps the protected part of the
    // tiles in flight (NP / kparts tiles of 128 rows) within 70 % of L2.
    int keep_pct = sched.l2_keep;
    if (keep_pct <= 0) {
        int dev = 0, l2 = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
        const double inflight = (double)NP / kparts * 128.0 * (double)ps.d * 2.0;
        keep_pct = (int)std::min(100.0, 100.0 * 0.7 * (double)l2 / std::max(inflight, 1.0));
        keep_pct = std::max(keep_pct, 1);
    }
    const int kkeep = ps.nk - (int)(((int64_t)ps.nk * std::min(keep_pct, 100) + 99) / 100);
    if (window < 1) window = 1;
    const int grid = NP > Dt2 * Sg ? NP : Dt2 * Sg;
    const uint32_t b_piece = (uint32_t)ps.m_pad * 128u;
    const uint32_t p_stage = 128u * 128u + b_piece, c_stage = 4u * 64u * 128u + b_piece;
    const int c_stages = 2;
    int p_stages = (int)((kSmemBudget - 2048 - c_stages * c_stage) / p_stage);
    if (p_stages > kMaxStages) p_stages = kMaxStages;
    if (p_stages < 2) return cudaErrorInvalidValue;
    const size_t smem =
        1024 + (size_t)p_stages * p_stage + (size_t)c_stages * c_stage + sizeof(FusedHeader);
    e = smem_at_least(reinterpret_cast<const void*>(xpass_fused_kernel), smem);
    if (e != cudaSuccess) return e;
    int* ready = sc.flags;
    int* consumed = sc.flags + ps.ntiles + 1;
    int* arrive = sc.flags + 2 * (ps.ntiles + 1);          // [tile][row quarter]
    int* pready = arrive + 4 * (ps.ntiles + 1);
    e = cudaMemsetAsync(sc.flags, 0, (size_t)(kparts == 2 ? 10 : 2) * (ps.ntiles + 1) * sizeof(int), st);
    // FP32 partials of the first K half, [tile][m_pad][128], after the BF16 Y^T in the Y scratch
    float* Ypart = reinterpret_cast<float*>(static_cast<__nv_bfloat16*>(sc.yt) + (size_t)ps.m_pad * ps.ldy);
    if (e != cudaSuccess) return e;
    // Consumer rows per TMEM accumulation before the fold into the double-float
    // partials (sched.flush 64-row K-stages).  A fold stalls the consumer's MMAs
    // (one accumulator set), so by default it happens every 2048 tiles (262144
    // rows): the FP32 tensor-core drift (about 2e-8 per accumulated MMA, 8 MMAs
    // per tile) stays below 4e-4 relative, far under the BF16 rounding of V and Y
    // that the fast pass carries anyway (2^-9).
    const int flush_tiles = sched.flush > 0 ? std::max(1, sched.flush / 2) : 2048;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kFusedThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    note_launch();
    e = cudaLaunchKernelEx(&cfg, xpass_fused_kernel, tmXa, tmV, tmXb, tmY, ps.ntiles, ps.nk, Dt2, Sg, NP, window,
                           flush_tiles, ps.m_pad, p_stages, c_stages, static_cast<__nv_bfloat16*>(sc.yt), ps.ldy,
                           static_cast<float*>(sc.zacc), ready, consumed, kparts, Ypart, arrive, pready, kkeep, status);
    if (e != cudaSuccess) return e;
    return launch_zreduce(static_cast<float*>(sc.zacc), Sg, 2 * Dt2, ps.d, m, ps.m_pad, Z, st);
}

// FP32 data: 3xTF32 passes (two kernels; X read twice).
cudaError_t run_pass_f32(const XView& x, const float* V, int m, int64_t r0, int64_t r1, float* Z, int flush,
                         const TcPassScratch& sc, int* status, int num_sms, cudaStream_t st,
                         const int64_t* row0_dev = nullptr) {
    const int64_t d = x.d, rows = r1 - r0;
    const int m_pad = m_pad_of(m);
    const int64_t ldv4 = round_up(d, 4);
    const int64_t ldy = round_up(rows, 128);
    const int Dt = (int)((d + 127) / 128);
    const int ntiles = (int)(ldy / 128), nk = (int)((d + kBK32 - 1) / kBK32);
    float* Vp = static_cast<float*>(sc.vp);
    float* Yt = static_cast<float*>(sc.yt);
    float* Zacc = static_cast<float*>(sc.zacc);
    {
        const int64_t total = (int64_t)m_pad * ldv4;
        int blocks = (int)((total + 255) / 256);
        if (blocks > 4096) blocks = 4096;
        note_launch();
        split_v_f32_kernel<<<blocks, 256, 0, st>>>(V, d, m, m_pad, ldv4, Vp);
    }
    // row0_dev (device, may be NULL): the batch's first row, read by the kernels
    const void* xbase = static_cast<const char*>(x.ptr) + (row0_dev ? 0 : r0) * x.ld * 4;
    const uint64_t xrows = row0_dev ? (uint64_t)x.n : (uint64_t)rows;
    CUtensorMap tmX, tmXr, tmV, tmY;
    const CUtensorMapDataType f32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    if (!encode_2d(&tmX, f32, xbase, d, xrows, x.ld * 4, 32, 128, CU_TENSOR_MAP_SWIZZLE_128B) ||
        !encode_2d(&tmXr, f32, xbase, d, xrows, x.ld * 4, 32, 32, CU_TENSOR_MAP_SWIZZLE_NONE) ||
        !encode_2d(&tmV, f32, Vp, d, 2 * (uint64_t)m_pad, ldv4 * 4, 32, m_pad, CU_TENSOR_MAP_SWIZZLE_128B) ||
        !encode_2d(&tmY, f32, Yt, ldy, 2 * (uint64_t)m_pad, ldy * 4, 32, m_pad, CU_TENSOR_MAP_SWIZZLE_128B))
        return cudaErrorInvalidValue;
    cudaError_t e;
    {
        const uint32_t stage_bytes = 2u * 16384u + 2u * (uint32_t)m_pad * 128u;
        int stages = (int)((kSmemBudget - 2048) / stage_bytes);
        if (stages > kMaxStages) stages = kMaxStages;
        const size_t smem = 1024 + (size_t)stages * stage_bytes + sizeof(F32Header);
        e = smem_at_least(reinterpret_cast<const void*>(xv_f32_kernel), smem);
        if (e != cudaSuccess) return e;
        // few row tiles (a minibatch) and a long K: split K so that every SM has work
        int ksplit = 1;
        if (ntiles * 2 <= num_sms && nk >= 8) {
            ksplit = (2 * num_sms + ntiles - 1) / ntiles;
            ksplit = std::min(ksplit, nk / 4);
            const int64_t cap = (int64_t)(sc.z_bytes / ((size_t)ldy * m_pad * sizeof(float)));
            ksplit = (int)std::min<int64_t>(ksplit, cap);
            if (ksplit < 2) ksplit = 1;
        }
        const int ntask = ntiles * ksplit;
        const int grid = ntask < num_sms ? ntask : num_sms;
        float* Ypart = static_cast<float*>(sc.zacc);
        note_launch();
        xv_f32_kernel<<<grid, kF32Threads, smem, st>>>(tmX, tmV, ntiles, nk, m_pad, stages, Yt, ldy, ksplit, Ypart,
                                                       status, row0_dev);
        if (ksplit > 1) {
            const int64_t total = ldy * m_pad;
            int blocks = (int)((total + 255) / 256);
            if (blocks > 4096) blocks = 4096;
            note_launch();
            ypart_reduce_f32_kernel<<<blocks, 256, 0, st>>>(Ypart, ksplit, ldy, m_pad, Yt);
        }
    }
    int Sg;
    {
        const uint32_t stage_bytes = 3u * 16384u + 2u * (uint32_t)m_pad * 128u;
        int stages = (int)((kSmemBudget - 2048) / stage_bytes);
        if (stages > kMaxStages) stages = kMaxStages;
        const size_t smem = 1024 + (size_t)stages * stage_bytes + sizeof(F32Header);
        e = smem_at_least(reinterpret_cast<const void*>(xty_f32_kernel), smem);
        if (e != cudaSuccess) return e;
        const int kst = (int)(ldy / kBK32);
        Sg = choose_row_groups(Dt, kst, num_sms, sc.z_bytes, m_pad);
        const int ntask = Dt * Sg;
        const int grid = ntask < num_sms ? ntask : num_sms;
        note_launch();
        xty_f32_kernel<<<grid, kF32Threads, smem, st>>>(tmXr, tmY, Dt, Sg, kst, flush, m_pad, stages, Zacc, status,
                                                        row0_dev);
    }
    return launch_zreduce(Zacc, Sg, Dt, d, m, m_pad, Z, st);
}

}  // namespace

size_t tc_pass_scratch_bytes(int64_t n, int64_t d, int m, int num_sms) {
    const Layout L = layout_of(n, d, m, num_sms);
    return L.vp_bytes + L.yt_bytes + L.z_bytes + L.flag_bytes + 4 * 256;
}

TcPassScratch tc_pass_scratch_carve(void* base, int64_t n, int64_t d, int m, int num_sms) {
    const Layout L = layout_of(n, d, m, num_sms);
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    TcPassScratch s;
    char* p = static_cast<char*>(base);
    s.vp = p;
    p += al(L.vp_bytes);
    s.yt = p;
    p += al(L.yt_bytes);
    s.zacc = p;
    s.z_bytes = L.z_bytes;
    p += al(L.z_bytes);
    s.flags = reinterpret_cast<int*>(p);
    return s;
}

bool tc_pass_supported(const XView& x, int m) {
    return (x.dtype == PPCA_BF16 || x.dtype == PPCA_F32 || x.dtype == PPCA_FP8_E4M3) && m >= 1 && m <= kMaxM &&
           encode_fn() != nullptr;
}

cudaError_t xpass_tc(const XView& x, const float* V, int m, int64_t r0, int64_t r1, float* Z, ppca_precision prec,
                     const TcPassScratch& s, const TcSchedule& sched, int* status, int num_sms, cudaStream_t st,
                     const int64_t* row0_dev) {
    if (r1 <= r0) return cudaErrorInvalidValue;
    if (row0_dev) {
        // device-side first row: whole 128-row tiles of FP32 or BF16 data, two-kernel forms
        if ((r1 - r0) % 128 != 0 || x.dtype == PPCA_FP8_E4M3) return cudaErrorInvalidValue;
        if (x.dtype == PPCA_F32) return run_pass_f32(x, V, m, r0, r1, Z, 64, s, status, num_sms, st, row0_dev);
        if (prec == PPCA_PREC_ACCURATE) return run_pass<3>(x, V, m, r0, r1, Z, 32, s, status, num_sms, st, row0_dev);
        return run_pass<1>(x, V, m, r0, r1, Z, 256, s, status, num_sms, st, row0_dev);
    }
    if (x.dtype == PPCA_F32) return run_pass_f32(x, V, m, r0, r1, Z, 64, s, status, num_sms, st);   // FAST only
    if (x.dtype == PPCA_FP8_E4M3) {
        if (prec == PPCA_PREC_ACCURATE) return run_pass<3, true>(x, V, m, r0, r1, Z, 32, s, status, num_sms, st);
        // the FP8 tensor cores when every SM gets row tiles (else the widening two-kernel pass, which splits K)
        const int64_t ntiles = (r1 - r0 + 127) / 128;
        if (sched.fp8_mma != 0 && ntiles * 2 > num_sms)
            return run_pass_f8(x, V, m, r0, r1, Z, 128, s, status, num_sms, st);
        return run_pass<1, true>(x, V, m, r0, r1, Z, 256, s, status, num_sms, st);
    }
    if (prec == PPCA_PREC_ACCURATE) return run_pass<3>(x, V, m, r0, r1, Z, 32, s, status, num_sms, st);
    // The fused pass needs every 128-column slice of d owned by a resident CTA.
    const int Dt = (int)((x.d + 127) / 128);
    const bool can_fuse = (Dt + 1) / 2 <= num_sms && (r1 - r0) >= 128 * 4;
    const bool fuse = sched.fused != 0 && can_fuse;
    if (fuse) return run_fused(x, V, m, r0, r1, Z, s, sched, status, num_sms, st);
    return run_pass<1>(x, V, m, r0, r1, Z, 256, s, status, num_sms, st);
}

bool xpass_tc_row0_same(const XView& x, int64_t rows, ppca_precision prec, const TcSchedule& sched, int num_sms) {
    if (rows % 128 != 0 || x.dtype == PPCA_FP8_E4M3) return false;
    if (x.dtype == PPCA_F32 || prec == PPCA_PREC_ACCURATE) return true;
    const int Dt = (int)((x.d + 127) / 128);
    const bool can_fuse = (Dt + 1) / 2 <= num_sms && rows >= 128 * 4;
    return !(sched.fused != 0 && can_fuse);
}

bool grouped_encode_maps(const GInst& g, GMaps& out) {
    const void* X = g.X;
    return encode_bf16_2d(&out.xa, X, g.d, g.n, g.ld * 2, 64, 128) &&
           encode_bf16_2d(&out.v, g.Vp, g.d, (uint64_t)g.m_pad, g.ldv * 2, 64, g.m_pad) &&
           encode_bf16_2d(&out.xb, X, g.d, g.n, g.ld * 2, 64, 64) &&
           encode_bf16_2d(&out.y, g.Yt, g.ldy, (uint64_t)g.m_pad, g.ldy * 2, 64, g.m_pad);
}

cudaError_t grouped_split_q(const GInst* gi, GTable blocks, cudaStream_t st) {
    note_launch();
    split_q_grouped_kernel<<<blocks.total, 256, 0, st>>>(gi, blocks);
    return cudaGetLastError();
}

cudaError_t grouped_xpass(const GInst* gi, const GMaps* maps, GTable xv_items, GTable xty_items, GTable zred_blocks,
                          int* status, int num_sms, cudaStream_t st) {
    const uint32_t xv_stage = 128u * 128u + 128u * 128u;
    const int xv_stages = stages_for(xv_stage);
    const size_t xv_smem = smem_bytes(xv_stages, xv_stage);
    cudaError_t e = smem_at_least(reinterpret_cast<const void*>(xv_grouped_kernel), xv_smem);
    if (e != cudaSuccess) return e;
    note_launch();
    xv_grouped_kernel<<<std::min(xv_items.total, num_sms), kThreads, xv_smem, st>>>(gi, maps, xv_items, xv_stages,
                                                                                   status);
    const uint32_t xty_stage = 2u * 64u * 128u + 128u * 128u;
    const int xty_stages = stages_for(xty_stage);
    const size_t xty_smem = smem_bytes(xty_stages, xty_stage);
    e = smem_at_least(reinterpret_cast<const void*>(xty_grouped_kernel), xty_smem);
    if (e != cudaSuccess) return e;
    note_launch();
    xty_grouped_kernel<<<std::min(xty_items.total, num_sms), kThreads, xty_smem, st>>>(gi, maps, xty_items, 256,
                                                                                      xty_stages, status);
    note_launch();
    zreduce_grouped_kernel<<<zred_blocks.total, 256, 0, st>>>(gi, zred_blocks);
    return cudaGetLastError();
}

cudaError_t pass_tc_set_wait_limit(uint64_t ns) { return tc::set_wait_limit(ns); }

}  // namespace ppca
