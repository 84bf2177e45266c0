// pass_gram.cu -- projected Gram matrix of the pPCA step on tcgen05 + TMA.
//
// Algorithm 1, steps 3-4 diagonalise the m x m matrix Q^T X^T X Q of an
// orthonormal Q (Section 3: the full PCA of the data projected on span(V)).
// It is formed as the Gram matrix of Y = X Q, so the pass over X runs one
// n x d x m contraction instead of the two of Z = X^T (X Q):
//
//   ygen   Y = X Q    persistent over 128-row tiles of X.  Q (FP32) is split
//                     into NV BF16 pieces; FP32 X is split in shared memory
//                     into NX BF16 pieces by eight transform warps (BF16 X is
//                     one exact piece).  Of the piece products x_a q_b those
//                     with a + b < max(NX, NV) are kept; the dropped ones are
//                     below 2^-24 of the result.
//   gram   G = Y^T Y  from Y's three BF16 pieces, products y_a^T y_b with
//                     a + b <= 2, one partial per CTA (FP32 pairs, second 0).
//   reduce G = sum of the partials in FP64, symmetrised.
//
// Accumulation.  An FP32 tensor-core accumulator that takes many MMAs in a row
// drifts: on sm_103a a relative error of roughly 2e-8 per accumulating MMA was
// measured, systematic rather than random, so it grows linearly with K, relative
// to the accumulator's own size.  In split precision both kernels therefore
// keep the product of the two leading pieces in an accumulator of its own,
// emptied every `flush` K-stages (64 wide) into an FP32 running sum in TMEM
// (which caps its drift at the MMAs of one flush group), and the products of
// the smaller pieces, at most 2^-8 of the result, in a second accumulator that
// is read once: its drift is relative to that smaller sum.  The FAST forms
// (one or three products) fold, if at all, into a double-float running sum.
//
// Warp roles: warp 0 issues TMA, warp 1 owns TMEM and issues the MMAs (one
// thread), warps 2-5 are the epilogue (TMEM lane quarter = warp % 4), warps
// 6-13 (FP32 X only) make the X pieces.  Every wait is bounded (2 s); on a
// timeout the kernel records kDevWaitTimeout, drains its copies, frees TMEM
// and returns.
#include <cudaTypedefs.h>

#include "grouped.h"
#include "pass_tc.h"
#include "tc_host.h"
#include "tc_ptx.cuh"

namespace ppca {

namespace {

constexpr int kGThreadsBf16 = 192;
constexpr int kGThreadsF32 = 448;             // + two groups of four transform warps
constexpr int kGMaxStages = 6;
constexpr int kGBK = 64;                    // K extent of one stage (64 BF16 = 128 B)
constexpr uint32_t kPiece = 128u * 128u;    // one 128-row x 128-byte operand tile
constexpr int kGSmemBudget = 227 * 1024;       // the opt-in maximum per block

struct GHeader {
    uint64_t full[kGMaxStages], xform[kGMaxStages], empty[kGMaxStages];
    uint64_t tfull[2], tempty[2];
    uint64_t bempty;                // split accumulation: the tile's small-piece sum has been read
    uint64_t drain;                 // the MMA thread's completion barrier after an abort
    uint32_t tmem_base;
    int abort;
    int xform_go[2];
};

__host__ __device__ inline uint32_t pow2_cols(uint32_t need) {
    uint32_t c = 32;
    while (c < need) c <<= 1;
    return c;
}

__device__ inline uint8_t* align1024(uint8_t* p) {
    return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

__device__ inline void g_prologue(GHeader* hd, int stages, uint32_t tmem_cols, const CUtensorMap* m0,
                                  const CUtensorMap* m1) {
    if (threadIdx.x == 0) {
        for (int i = 0; i < stages; ++i) {
            tc::mbar_init(&hd->full[i], 1);
            tc::mbar_init(&hd->xform[i], 128);
            tc::mbar_init(&hd->empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&hd->tfull[i], 1);
            tc::mbar_init(&hd->tempty[i], 128);
        }
        tc::mbar_init(&hd->bempty, 128);
        tc::mbar_init(&hd->drain, 1);
        hd->abort = 0;
        hd->xform_go[0] = hd->xform_go[1] = 0;
        tc::mbar_init_fence();
        tc::tma_prefetch(m0);
        if (m1) tc::tma_prefetch(m1);
    }
    if (threadIdx.x / 32 == 1) tc::tmem_alloc(&hd->tmem_base, tmem_cols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

// After an abort the MMA thread (warp 1, lane 0) first waits for its MMAs.
__device__ inline void g_teardown(GHeader* hd, uint32_t tmem_cols, int* status) {
    if (threadIdx.x == 32 && *(volatile int*)&hd->abort) tc::drain_mmas(&hd->drain, status);
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x / 32 == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(hd->tmem_base, tmem_cols);
    }
}

__device__ inline void g_drain(GHeader* hd, uint32_t issued, int stages, int* status) {
    const uint32_t first = issued > (uint32_t)stages ? issued - (uint32_t)stages : 0u;
    for (uint32_t it = first; it < issued; ++it)
        tc::mbar_wait(&hd->full[it % stages], (it / stages) & 1u, status, 100000000ull);
}

// (hi, lo) -> three BF16 pieces whose sum is hi + lo to about 2^-24.
__device__ __forceinline__ void split3_df(float hi, float lo, __nv_bfloat16* dst, int64_t piece_stride) {
    const __nv_bfloat16 p1 = __float2bfloat16_rn(hi);
    const float r1 = __fadd_rn(__fsub_rn(hi, __bfloat162float(p1)), lo);
    const __nv_bfloat16 p2 = __float2bfloat16_rn(r1);
    const float r2 = __fsub_rn(r1, __bfloat162float(p2));
    dst[0] = p1;
    dst[piece_stride] = p2;
    dst[2 * piece_stride] = __float2bfloat16_rn(r2);
}

// One flush group's epilogue step for a 32-column chunk of this thread's TMEM
// lane: fold the accumulator chunk `a` into the running sum (R, L) at column
// offset `run`; returns the updated sum in (rh, rl).  g = group index.
__device__ __forceinline__ void fold_chunk(uint32_t lane_base, uint32_t acc_col, uint32_t run_col, uint32_t lo_off,
                                           int g, bool keep, uint32_t (&a)[32], uint32_t (&rh)[32],
                                           uint32_t (&rl)[32]) {
    tc::tmem_ld32(lane_base + acc_col, a);
    if (g == 0) {
        tc::tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            rh[j] = a[j];
            rl[j] = 0u;
        }
    } else {
        tc::tmem_ld32(lane_base + run_col, rh);
        tc::tmem_ld32(lane_base + run_col + lo_off, rl);
        tc::tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            float hi = __uint_as_float(rh[j]), lo = __uint_as_float(rl[j]);
            df_add(hi, lo, __uint_as_float(a[j]));
            rh[j] = __float_as_uint(hi);
            rl[j] = __float_as_uint(lo);
        }
    }
    if (keep) {
        tc::tmem_st32(lane_base + run_col, rh);
        tc::tmem_st32(lane_base + run_col + lo_off, rl);
        tc::tmem_st_wait();
    }
}

// ---------------------------------------------------------------- Y = X Q

// One 128-row tile of Y = X Q: the descriptors of X and of the Q pieces, the
// first X row, the K-stages, the basis width (the MMA's N) and where its rows
// of the Y pieces go (piece p at Yt + p m_pad ldy, transposed).
struct YItem {
    const CUtensorMap* mx;
    const CUtensorMap* mq;
    int xr;
    int nk;
    int m_pad;
    __nv_bfloat16* Yt;
    int64_t ldy;
    int64_t row;
};

// One problem: tile t of rows [r0, r1), or the t-th listed 128-row block.
struct YgenOne {
    CUtensorMap tmX, tmQ;
    int ntiles, nk, m_pad;
    __nv_bfloat16* Yt;
    int64_t ldy;
    const int* tile_row;
    __device__ int count() const { return ntiles; }
    __device__ YItem item(int t) const {
        return YItem{&tmX, &tmQ, tile_row ? tile_row[t] : t * 128, nk, m_pad, Yt, ldy, (int64_t)t * 128};
    }
};

// Many problems (grouped.h): item w is tile w - base[i] of instance i.
struct YgenGroup {
    const GInst* gi;
    const GMaps* maps;
    GTable items;
    __device__ int count() const { return items.total; }
    __device__ YItem item(int w) const {
        const int i = group_find(items, w), t = w - items.base[i];
        const GInst& g = gi[i];
        return YItem{&maps[i].xp, &maps[i].q3, t * 128, g.nk, g.m_pad, g.Y3, g.ldy, (int64_t)t * 128};
    }
};

// Stage: [X area][Q piece 0 .. NV-1], pieces q_piece bytes apart.  X area: BF16
// X -> one 16 KB tile; FP32 X -> two raw 32-column boxes (32 KB), overwritten in
// place by the NX pieces.
//
// Accumulation.  FAST (one or three products, no fold): accumulator b at TMEM
// column b * acc_stride, the double-float running sum at [2, 4) * acc_stride.
// Split precision (NV = 3): the leading product x_0 q_0 goes to accumulator b,
// emptied every `flush` K-stages into an FP32 running sum R (column 2
// acc_stride); the other products, at most 2^-8 of Y, go to one accumulator S
// (column 3 acc_stride) for the whole tile: an accumulator drifts relative to
// its own size, so S needs no fold, and a fold of the leading product alone is
// a load, an add and a store.  Y = (R + acc_last) + S.
template <int NX, int NV, bool F32X, class Work>
__global__ void __launch_bounds__(F32X ? kGThreadsF32 : kGThreadsBf16, 1)
    ygen_kernel(const __grid_constant__ Work work, int flush, int stages, uint32_t q_piece, uint32_t acc_stride,
                uint32_t tmem_cols, int* status) {
    constexpr int ORD = (NX > NV ? NX : NV) - 1;
    constexpr bool SPLIT = NV == 3;
    constexpr uint32_t x_bytes = F32X ? (NX > 2 ? NX : 2) * kPiece : kPiece;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* tiles = align1024(smem_raw);
    const uint32_t stage_bytes = x_bytes + NV * q_piece;
    GHeader* hd = reinterpret_cast<GHeader*>(tiles + (size_t)stages * stage_bytes);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    {
        const YItem first = work.item(0);
        g_prologue(hd, stages, tmem_cols, first.mx, first.mq);
    }
    const uint32_t tmem = hd->tmem_base;
    volatile int* abort_flag = &hd->abort;
    const int count = work.count();

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            for (int w = blockIdx.x; w < count && ok; w += gridDim.x) {
                const YItem y = work.item(w);
                const uint32_t q_bytes = (uint32_t)y.m_pad * 128u;
                for (int k = 0; k < y.nk; ++k, ++it) {
                    const uint32_t s = it % stages, ph = (it / stages) & 1u;
                    if (!tc::mbar_wait(&hd->empty[s], ph ^ 1u, status) || *abort_flag) {
                        *abort_flag = 1;
                        ok = false;
                        break;
                    }
                    tc::mbar_expect_tx(&hd->full[s], (F32X ? 2u * kPiece : kPiece) + NV * q_bytes);
                    uint8_t* st = tiles + (size_t)s * stage_bytes;
                    if (F32X) {
                        tc::tma_load_2d(st, y.mx, &hd->full[s], k * kGBK, y.xr);
                        tc::tma_load_2d(st + kPiece, y.mx, &hd->full[s], k * kGBK + 32, y.xr);
                    } else {
                        tc::tma_load_2d(st, y.mx, &hd->full[s], k * kGBK, y.xr);
                    }
#pragma unroll
                    for (int p = 0; p < NV; ++p)
                        tc::tma_load_2d(st + x_bytes + p * q_piece, y.mq, &hd->full[s], k * kGBK, p * y.m_pad);
                }
            }
            if (!ok) g_drain(hd, it, stages, status);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            uint32_t it = 0, fb = 0, tl = 0;
            bool ok = true;
            for (int w = blockIdx.x; w < count && ok; w += gridDim.x, ++tl) {
                const YItem y = work.item(w);
                const uint32_t idesc = tc::idesc_bf16(128, y.m_pad, false, false);
                const int ngroups = (y.nk + flush - 1) / flush;
                const uint32_t s_tmem = tmem + 3u * acc_stride;
                uint32_t acc_s = 0;
                if (SPLIT) {
                    // the previous tile's small-piece sum must have been read
                    if (!tc::mbar_wait(&hd->bempty, (tl & 1u) ^ 1u, status) || *abort_flag) {
                        *abort_flag = 1;
                        break;
                    }
                    tc::fence_after_sync();
                }
                for (int g = 0; g < ngroups && ok; ++g, ++fb) {
                    const uint32_t b = fb & 1u, tph = (fb >> 1) & 1u;
                    if (!tc::mbar_wait(&hd->tempty[b], tph ^ 1u, status) || *abort_flag) {
                        *abort_flag = 1;
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t d_tmem = tmem + b * acc_stride;
                    const int k0 = g * flush, k1 = k0 + flush < y.nk ? k0 + flush : y.nk;
                    uint32_t acc = 0;
                    for (int k = k0; k < k1; ++k, ++it) {
                        const uint32_t s = it % stages, ph = (it / stages) & 1u;
                        if (!tc::mbar_wait(F32X ? &hd->xform[s] : &hd->full[s], ph, status) || *abort_flag) {
                            *abort_flag = 1;
                            ok = false;
                            break;
                        }
                        tc::fence_after_sync();
                        const uint32_t a0 = tc::smem_u32(tiles + (size_t)s * stage_bytes);
#pragma unroll
                        for (int kk = 0; kk < kGBK / 16; ++kk) {
#pragma unroll
                            for (int pa = 0; pa < NX; ++pa) {
#pragma unroll
                                for (int pb = 0; pb < NV; ++pb) {
                                    if (pa + pb > ORD) continue;
                                    const uint64_t ad = tc::smem_desc_sw128(a0 + pa * kPiece + kk * 32, 16, 1024);
                                    const uint64_t bd =
                                        tc::smem_desc_sw128(a0 + x_bytes + pb * q_piece + kk * 32, 16, 1024);
                                    if (SPLIT && (pa | pb) != 0) {
                                        tc::mma_f16(s_tmem, ad, bd, idesc, acc_s);
                                        acc_s = 1;
                                    } else {
                                        tc::mma_f16(d_tmem, ad, bd, idesc, acc);
                                        acc = 1;
                                    }
                                }
                            }
                        }
                        tc::mma_commit(&hd->empty[s]);
                    }
                    if (ok) tc::mma_commit(&hd->tfull[b]);
                }
            }
        }
    } else if (warp < 6) {
        const int q = warp & 3;
        const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
        uint32_t fb = 0;
        bool ok = true;
        for (int w = blockIdx.x; w < count && ok; w += gridDim.x) {
            const YItem y = work.item(w);
            const int64_t row = y.row + q * 32 + lane;
            const int64_t piece_stride = (int64_t)y.m_pad * y.ldy;
            const int ngroups = (y.nk + flush - 1) / flush;
            for (int g = 0; g < ngroups; ++g, ++fb) {
                const uint32_t b = fb & 1u, tph = (fb >> 1) & 1u;
                if (!tc::mbar_wait(&hd->tfull[b], tph, status) || *abort_flag) {
                    *abort_flag = 1;
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                const bool last = g == ngroups - 1;
                for (int c0 = 0; c0 < y.m_pad; c0 += 32) {
                    if (SPLIT) {
                        const uint32_t a_col = b * acc_stride + (uint32_t)c0, r_col = 2u * acc_stride + (uint32_t)c0;
                        uint32_t a[32], r[32];
                        tc::tmem_ld32(lane_base + a_col, a);
                        if (g > 0) tc::tmem_ld32(lane_base + r_col, r);
                        tc::tmem_ld_wait();
                        if (g > 0) {
#pragma unroll
                            for (int j = 0; j < 32; ++j) a[j] = __float_as_uint(__uint_as_float(r[j]) + __uint_as_float(a[j]));
                        }
                        if (!last) {
                            tc::tmem_st32(lane_base + r_col, a);
                            tc::tmem_st_wait();
                        } else {
                            tc::tmem_ld32(lane_base + 3u * acc_stride + (uint32_t)c0, r);
                            tc::tmem_ld_wait();
#pragma unroll
                            for (int j = 0; j < 32; ++j)
                                split3_df(__uint_as_float(a[j]) + __uint_as_float(r[j]), 0.f,
                                          y.Yt + (int64_t)(c0 + j) * y.ldy + row, piece_stride);
                        }
                    } else {
                        uint32_t a[32], rh[32], rl[32];
                        fold_chunk(lane_base, b * acc_stride + (uint32_t)c0, 2u * acc_stride + (uint32_t)c0,
                                   acc_stride, g, !last, a, rh, rl);
                        if (last) {
#pragma unroll
                            for (int j = 0; j < 32; ++j)
                                split3_df(__uint_as_float(rh[j]), __uint_as_float(rl[j]),
                                          y.Yt + (int64_t)(c0 + j) * y.ldy + row, piece_stride);
                        }
                    }
                }
                tc::fence_before_sync();
                tc::mbar_arrive(&hd->tempty[b]);
                if (SPLIT && last) tc::mbar_arrive(&hd->bempty);
            }
        }
    } else if (F32X) {
        // Raw FP32 (two boxes of 128 rows x 32 columns, 128-byte swizzle) ->
        // NX BF16 pieces (128 rows x 64 columns, 128-byte swizzle), in place.
        // Task (r, c): row r, piece chunk c = columns 8c .. 8c+7 = raw box c / 4,
        // raw chunks 2 (c % 4) and 2 (c % 4) + 1.  Two groups of four warps take
        // the even and the odd stages, so two stages are split at once.
        const int grp = (warp - 6) / 4;
        const int tid = threadIdx.x - 192 - grp * 128;
        uint32_t it = 0;
        bool ok = true;
        for (int w = blockIdx.x; w < count && ok; w += gridDim.x) {
            const int nk = work.item(w).nk;
            for (int k = 0; k < nk; ++k, ++it) {
                if ((int)(it & 1u) != grp) continue;
                const uint32_t s = it % stages, ph = (it / stages) & 1u;
                if (tid == 0) {
                    const bool go = tc::mbar_wait(&hd->full[s], ph, status) && !*abort_flag;
                    if (!go) *abort_flag = 1;
                    *(volatile int*)&hd->xform_go[grp] = go ? 1 : 0;
                }
                tc::named_barrier(1 + grp, 128);
                if (!*(volatile int*)&hd->xform_go[grp]) {
                    ok = false;
                    break;
                }
                uint8_t* xs = tiles + (size_t)s * stage_bytes;
                float v[8][8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int id = i * 128 + tid, r = id >> 3, c = id & 7;
                    const uint8_t* rowp = xs + (c >> 2) * kPiece + r * 128;
                    const int q0 = (c & 3) * 2;
                    const float4 u0 = *reinterpret_cast<const float4*>(rowp + ((q0 ^ (r & 7)) << 4));
                    const float4 u1 = *reinterpret_cast<const float4*>(rowp + (((q0 + 1) ^ (r & 7)) << 4));
                    v[i][0] = u0.x; v[i][1] = u0.y; v[i][2] = u0.z; v[i][3] = u0.w;
                    v[i][4] = u1.x; v[i][5] = u1.y; v[i][6] = u1.z; v[i][7] = u1.w;
                }
                tc::named_barrier(1 + grp, 128);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int id = i * 128 + tid, r = id >> 3, c = id & 7;
                    uint32_t wd[NX][4];
#pragma unroll
                    for (int e = 0; e < 8; e += 2) {
                        float x0 = v[i][e], x1 = v[i][e + 1];
#pragma unroll
                        for (int p = 0; p < NX; ++p) {
                            // both values rounded to nearest by one paired conversion (x0 low)
                            const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
                            wd[p][e / 2] = *reinterpret_cast<const uint32_t*>(&h);
                            const float2 hf = __bfloat1622float2(h);
                            x0 = __fsub_rn(x0, hf.x);
                            x1 = __fsub_rn(x1, hf.y);
                        }
                    }
                    const uint32_t off = (uint32_t)r * 128u + (uint32_t)((c ^ (r & 7)) << 4);
#pragma unroll
                    for (int p = 0; p < NX; ++p)
                        *reinterpret_cast<uint4*>(xs + p * kPiece + off) =
                            make_uint4(wd[p][0], wd[p][1], wd[p][2], wd[p][3]);
                }
                tc::fence_proxy_async_shared();
                tc::mbar_arrive(&hd->xform[s]);
            }
        }
    }
    g_teardown(hd, tmem_cols, status);
}

// ---------------------------------------------------------------- G = Y^T Y

// One CTA's share of G = Y^T Y: K-stages [k0, k1) of the Y pieces (descriptor
// my, basis width m_pad), written as an m_pad x m_pad double-float partial.
struct GramItem {
    const CUtensorMap* my;
    int k0, k1, m_pad;
    float2* part;
};

// One problem: CTA c takes K-stages [c kst / grid, (c + 1) kst / grid).
struct GramOne {
    CUtensorMap tmY;
    int kst, m_pad;
    float2* parts;
    __device__ GramItem item(int c) const {
        return GramItem{&tmY, (int)((int64_t)c * kst / gridDim.x), (int)((int64_t)(c + 1) * kst / gridDim.x), m_pad,
                        parts + (int64_t)c * m_pad * m_pad};
    }
};

// Many problems: CTA c is chunk c - base[i] (kGramChunk K-stages) of instance i.
struct GramGroup {
    const GInst* gi;
    const GMaps* maps;
    GTable items;
    __device__ GramItem item(int c) const {
        const int i = group_find(items, c), p = c - items.base[i];
        const GInst& g = gi[i];
        const int kst = (int)(g.ldy / kGBK);
        const int k0 = p * kGramChunk, k1 = k0 + kGramChunk < kst ? k0 + kGramChunk : kst;
        return GramItem{&maps[i].y3, k0, k1, g.m_pad, g.Gpart + (int64_t)p * g.m_pad * g.m_pad};
    }
};

// Stage: three 16 KB slots (pieces y1, y2, y3 of 64 rows of Y, as m_pad rows of
// Y^T x 128 B); slot rows m_pad .. 127 stay zero so the M = 128 MMA reads
// zeros there.  Every CTA has at least one K-stage.  Accumulation as in
// ygen's split precision: y1^T y1 in accumulator b (TMEM column b m_pad),
// emptied every `flush` K-stages into an FP32 running sum (column 2 m_pad);
// the five smaller products in one accumulator (column 3 m_pad) for the CTA's
// whole K range.
template <class Work>
__global__ void __launch_bounds__(kGThreadsBf16, 1)
    gram_y_kernel(const __grid_constant__ Work work, int flush, int stages, int* status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* tiles = align1024(smem_raw);
    const uint32_t stage_bytes = 3u * kPiece;
    GHeader* hd = reinterpret_cast<GHeader*>(tiles + (size_t)stages * stage_bytes);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const GramItem gw = work.item(blockIdx.x);
    const int k0 = gw.k0, k1 = gw.k1, m_pad = gw.m_pad;
    const int ngroups = (k1 - k0 + flush - 1) / flush;
    const uint32_t tmem_cols = pow2_cols(4u * (uint32_t)m_pad);
    // zero the slot rows no TMA box covers
    {
        const uint32_t tail = (128u - (uint32_t)m_pad) * 128u / 16u;   // uint4 per slot
        for (uint32_t e = threadIdx.x; e < (uint32_t)stages * 3u * tail; e += blockDim.x) {
            const uint32_t slot = e / tail, w = e % tail;
            *reinterpret_cast<uint4*>(tiles + slot * kPiece + (uint32_t)m_pad * 128u + w * 16u) =
                make_uint4(0u, 0u, 0u, 0u);
        }
        tc::fence_proxy_async_shared();
    }
    g_prologue(hd, stages, tmem_cols, gw.my, nullptr);
    const uint32_t tmem = hd->tmem_base;
    volatile int* abort_flag = &hd->abort;
    const uint32_t box_bytes = (uint32_t)m_pad * 128u;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;
            for (int k = k0; k < k1; ++k, ++it) {
                const uint32_t s = it % stages, ph = (it / stages) & 1u;
                if (!tc::mbar_wait(&hd->empty[s], ph ^ 1u, status) || *abort_flag) {
                    *abort_flag = 1;
                    g_drain(hd, it, stages, status);
                    break;
                }
                tc::mbar_expect_tx(&hd->full[s], 3u * box_bytes);
                uint8_t* st = tiles + (size_t)s * stage_bytes;
#pragma unroll
                for (int p = 0; p < 3; ++p) tc::tma_load_2d(st + p * kPiece, gw.my, &hd->full[s], k * kGBK, p * m_pad);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_bf16(128, m_pad, false, false);
            const uint32_t s_tmem = tmem + 3u * (uint32_t)m_pad;
            uint32_t it = 0, acc_s = 0;
            bool ok = true;
            for (int g = 0; g < ngroups && ok; ++g) {
                const uint32_t b = (uint32_t)g & 1u, tph = ((uint32_t)g >> 1) & 1u;
                if (!tc::mbar_wait(&hd->tempty[b], tph ^ 1u, status) || *abort_flag) {
                    *abort_flag = 1;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t d_tmem = tmem + b * (uint32_t)m_pad;
                const int ka = k0 + g * flush, kb = ka + flush < k1 ? ka + flush : k1;
                uint32_t acc = 0;
                for (int k = ka; k < kb; ++k, ++it) {
                    const uint32_t s = it % stages, ph = (it / stages) & 1u;
                    if (!tc::mbar_wait(&hd->full[s], ph, status) || *abort_flag) {
                        *abort_flag = 1;
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t a0 = tc::smem_u32(tiles + (size_t)s * stage_bytes);
#pragma unroll
                    for (int kk = 0; kk < kGBK / 16; ++kk) {
#pragma unroll
                        for (int pa = 0; pa < 3; ++pa) {
#pragma unroll
                            for (int pb = 0; pb < 3; ++pb) {
                                if (pa + pb > 2) continue;
                                const uint64_t ad = tc::smem_desc_sw128(a0 + pa * kPiece + kk * 32, 16, 1024);
                                const uint64_t bd = tc::smem_desc_sw128(a0 + pb * kPiece + kk * 32, 16, 1024);
                                if ((pa | pb) != 0) {
                                    tc::mma_f16(s_tmem, ad, bd, idesc, acc_s);
                                    acc_s = 1;
                                } else {
                                    tc::mma_f16(d_tmem, ad, bd, idesc, acc);
                                    acc = 1;
                                }
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
        const int i = q * 32 + lane;                 // row of G
        const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
        const bool live = q * 32 < m_pad;            // warp-uniform
        for (int g = 0; g < ngroups; ++g) {
            const uint32_t b = (uint32_t)g & 1u, tph = ((uint32_t)g >> 1) & 1u;
            if (!tc::mbar_wait(&hd->tfull[b], tph, status) || *abort_flag) {
                *abort_flag = 1;
                break;
            }
            tc::fence_after_sync();
            const bool last = g == ngroups - 1;
            if (live) {
                for (int c0 = 0; c0 < m_pad; c0 += 32) {
                    const uint32_t a_col = b * (uint32_t)m_pad + (uint32_t)c0, r_col = 2u * (uint32_t)m_pad + (uint32_t)c0;
                    uint32_t a[32], r[32];
                    tc::tmem_ld32(lane_base + a_col, a);
                    if (g > 0) tc::tmem_ld32(lane_base + r_col, r);
                    tc::tmem_ld_wait();
                    if (g > 0) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) a[j] = __float_as_uint(__uint_as_float(r[j]) + __uint_as_float(a[j]));
                    }
                    if (!last) {
                        tc::tmem_st32(lane_base + r_col, a);
                        tc::tmem_st_wait();
                    } else {
                        tc::tmem_ld32(lane_base + 3u * (uint32_t)m_pad + (uint32_t)c0, r);
                        tc::tmem_ld_wait();
                        float2* dst = gw.part + (int64_t)i * m_pad + c0;
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            dst[j] = make_float2(__uint_as_float(a[j]) + __uint_as_float(r[j]), 0.f);
                    }
                }
            }
            tc::fence_before_sync();
            tc::mbar_arrive(&hd->tempty[b]);
        }
    }
    g_teardown(hd, tmem_cols, status);
}

// G[i][j] = (sum_p part_p[i][j] + sum_p part_p[j][i]) / 2 in FP64.
__global__ void gram_parts_reduce_kernel(const float2* __restrict__ Gpart, int nparts, int m, int m_pad,
                                         double* __restrict__ G, float* __restrict__ Gf) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m * m) return;
    const int i = e / m, j = e % m;
    double s = 0.0;
    for (int p = 0; p < nparts; ++p) {
        const float2 a = Gpart[((int64_t)p * m_pad + i) * m_pad + j];
        const float2 b = Gpart[((int64_t)p * m_pad + j) * m_pad + i];
        s += ((double)a.x + (double)a.y) + ((double)b.x + (double)b.y);
    }
    G[e] = 0.5 * s;
    if (Gf) Gf[e] = (float)(0.5 * s);
}

// The grouped reduction: instance i's blocks reduce its nparts partials.
__global__ void gram_parts_reduce_grouped_kernel(const GInst* __restrict__ gi, GTable tab) {
    const int i = group_find(tab, blockIdx.x);
    const GInst& g = gi[i];
    const int e = (blockIdx.x - tab.base[i]) * blockDim.x + threadIdx.x;
    const int m = g.m, m_pad = g.m_pad;
    if (e >= m * m) return;
    const int r = e / m, c = e % m;
    double s = 0.0;
    for (int p = 0; p < g.nparts; ++p) {
        const float2 a = g.Gpart[((int64_t)p * m_pad + r) * m_pad + c];
        const float2 b = g.Gpart[((int64_t)p * m_pad + c) * m_pad + r];
        s += ((double)a.x + (double)a.y) + ((double)b.x + (double)b.y);
    }
    g.Gp[e] = 0.5 * s;
}

// ygen over `work` (count() items, each 128 rows): the Q-piece slots and the
// TMEM accumulators are laid out for the widest basis, m_pad_max; grid =
// min(items, SMs).
template <int NX, int NV, bool F32X, class Work>
cudaError_t launch_ygen(const Work& work, int items, int flush, int m_pad_max, int* status, int num_sms,
                        cudaStream_t st) {
    constexpr uint32_t x_bytes = F32X ? (NX > 2 ? NX : 2) * kPiece : kPiece;
    const uint32_t q_piece = (uint32_t)m_pad_max * 128u;
    const uint32_t stage_bytes = x_bytes + NV * q_piece;
    int stages = (int)((kGSmemBudget - 2048) / stage_bytes);
    if (stages > kGMaxStages) stages = kGMaxStages;
    if (stages < 2) return cudaErrorInvalidValue;
    const size_t smem = 1024 + (size_t)stages * stage_bytes + sizeof(GHeader);
    // accumulators: two buffers and the double-float running sum
    const uint32_t acc_stride = (uint32_t)m_pad_max;
    const uint32_t tmem_cols = pow2_cols(4u * acc_stride);
    auto kern = ygen_kernel<NX, NV, F32X, Work>;
    cudaError_t e = smem_at_least(reinterpret_cast<const void*>(kern), smem);
    if (e != cudaSuccess) return e;
    const int grid = items < num_sms ? items : num_sms;
    note_launch();
    kern<<<grid, F32X ? kGThreadsF32 : kGThreadsBf16, smem, st>>>(work, flush, stages, q_piece, acc_stride, tmem_cols,
                                                                 status);
    return cudaGetLastError();
}

template <class Work>
cudaError_t launch_gram_y(const Work& work, int grid, int* status, cudaStream_t st) {
    const int gstages = 4;
    const size_t smem = 1024 + (size_t)gstages * 3 * kPiece + sizeof(GHeader);
    auto kern = gram_y_kernel<Work>;
    cudaError_t e = smem_at_least(reinterpret_cast<const void*>(kern), smem);
    if (e != cudaSuccess) return e;
    note_launch();
    kern<<<grid, kGThreadsBf16, smem, st>>>(work, 12, gstages, status);
    return cudaGetLastError();
}

inline int64_t rup(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

}  // namespace

namespace {

// G = (X_S Q)^T (X_S Q) with X_S = rows [r0, r1) (tile_row == nullptr) or the
// nsel listed 128-row blocks of X (tile_row: device array of their first rows).
cudaError_t projected_gram_impl(const XView& x, const float* Q, int m, int64_t r0, int64_t r1,
                                const int* tile_row, int nsel, double* G, ppca_precision prec, int flush,
                                const TcPassScratch& sc, int* status, int num_sms, cudaStream_t st) {
    if (r1 <= r0 || m < 1 || m > 128) return cudaErrorInvalidValue;
    if (tile_row && nsel < 1) return cudaErrorInvalidValue;
    const bool f32 = x.dtype == PPCA_F32;
    const bool accurate = prec != PPCA_PREC_FAST;
    const int m_pad = (int)rup(m, 32);
    const int64_t d = x.d, rows = r1 - r0;
    const int64_t ldv = rup(d, 8), ldy = tile_row ? (int64_t)nsel * 128 : rup(rows, 128);
    const int ntiles = (int)(ldy / 128), nk = (int)((d + kGBK - 1) / kGBK);
    const int NV = accurate ? 3 : (f32 ? 2 : 1);
    // K-stages per fold of the leading product's FP32 tensor-core accumulator
    // into the running sum.  Each accumulating MMA adds ~2e-8 drift relative to
    // the accumulator: a fold every 12 stages lets it take 48 MMAs (4 per
    // stage), the drift the earlier all-products accumulator had at a fold every
    // 4 (BF16 X) or 2 (FP32 X) stages, at a twelfth of the folds.
    if (flush <= 0) flush = accurate ? 12 : nk;
    __nv_bfloat16* Qp = static_cast<__nv_bfloat16*>(sc.vp);
    __nv_bfloat16* Yt = static_cast<__nv_bfloat16*>(sc.yt);
    cudaError_t e = launch_split_v(Q, d, m, m_pad, ldv, NV, Qp, st);
    if (e != cudaSuccess) return e;
    CUtensorMap tmX, tmQ, tmY;
    const int esz = f32 ? 4 : 2;
    const void* xbase = static_cast<const char*>(x.ptr) + r0 * x.ld * esz;
    const bool ok_x = f32 ? encode_2d(&tmX, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, xbase, d, rows, x.ld * 4, 32, 128,
                                      CU_TENSOR_MAP_SWIZZLE_128B)
                          : encode_bf16_2d(&tmX, xbase, d, rows, x.ld * 2, 64, 128);
    if (!ok_x || !encode_bf16_2d(&tmQ, Qp, d, (uint64_t)NV * m_pad, ldv * 2, 64, m_pad) ||
        !encode_bf16_2d(&tmY, Yt, ldy, 3ull * m_pad, ldy * 2, 64, m_pad))
        return cudaErrorInvalidValue;
    YgenOne yw{tmX, tmQ, ntiles, nk, m_pad, Yt, ldy, tile_row};
    if (f32) {
        e = accurate ? launch_ygen<3, 3, true>(yw, ntiles, flush, m_pad, status, num_sms, st)
                     : launch_ygen<2, 2, true>(yw, ntiles, flush, m_pad, status, num_sms, st);
    } else {
        e = accurate ? launch_ygen<1, 3, false>(yw, ntiles, flush, m_pad, status, num_sms, st)
                     : launch_ygen<1, 1, false>(yw, ntiles, flush, m_pad, status, num_sms, st);
    }
    if (e != cudaSuccess) return e;
    // G = Y^T Y
    const int kst = (int)(ldy / kGBK);
    const int grid = kst < num_sms ? kst : num_sms;
    float2* parts = static_cast<float2*>(sc.zacc);
    e = launch_gram_y(GramOne{tmY, kst, m_pad, parts}, grid, status, st);
    if (e != cudaSuccess) return e;
    note_launch();
    gram_parts_reduce_kernel<<<(m * m + 255) / 256, 256, 0, st>>>(parts, grid, m, m_pad, G, nullptr);
    return cudaGetLastError();
}

}  // namespace

cudaError_t projected_gram_tc(const XView& x, const float* Q, int m, int64_t r0, int64_t r1, double* G,
                              ppca_precision prec, int flush, const TcPassScratch& sc, int* status, int num_sms,
                              cudaStream_t st) {
    return projected_gram_impl(x, Q, m, r0, r1, nullptr, 0, G, prec, flush, sc, status, num_sms, st);
}

cudaError_t projected_gram_tc_blocks(const XView& x, const float* Q, int m, const int* tile_row, int nsel, double* G,
                                     ppca_precision prec, int flush, const TcPassScratch& sc, int* status,
                                     int num_sms, cudaStream_t st) {
    return projected_gram_impl(x, Q, m, 0, x.n, tile_row, nsel, G, prec, flush, sc, status, num_sms, st);
}

// G = Z^T Z for a d x m column-major FP32 Z (CholeskyQR's Gram matrix) on the
// tensor cores: Z is split into three BF16 pieces (the layout of the projected
// Gram's Y pieces, K = d), G = sum over the six piece products with a + b <= 2
// (accumulated as in gram_y_kernel), one partial per CTA, summed and
// symmetrised in FP64; Gf receives the FP32 rounding of G.
cudaError_t gram_tc(const float* Z, int64_t d, int m, double* G, float* Gf, const TcPassScratch& sc, int* status,
                    int num_sms, cudaStream_t st) {
    if (m < 1 || m > 128 || d < 1) return cudaErrorInvalidValue;
    const int m_pad = (int)rup(m, 32);
    const int64_t ldv = rup(d, 8);
    __nv_bfloat16* Zp = static_cast<__nv_bfloat16*>(sc.vp);
    cudaError_t e = launch_split_v(Z, d, m, m_pad, ldv, 3, Zp, st);
    if (e != cudaSuccess) return e;
    CUtensorMap tmY;
    if (!encode_bf16_2d(&tmY, Zp, (uint64_t)d, 3ull * m_pad, ldv * 2, 64, m_pad)) return cudaErrorInvalidValue;
    const int kst = (int)((d + kGBK - 1) / kGBK);
    // eight K-stages per CTA: fewer double-float partials (m_pad^2 x 8 B each) to
    // write and sum; measured best of 1-16 at d = 16384 and 262144
    int grid = kst / 8;
    if (grid > num_sms) grid = num_sms;
    if (grid < 1) grid = 1;
    float2* parts = static_cast<float2*>(sc.zacc);
    e = launch_gram_y(GramOne{tmY, kst, m_pad, parts}, grid, status, st);
    if (e != cudaSuccess) return e;
    note_launch();
    gram_parts_reduce_kernel<<<(m * m + 255) / 256, 256, 0, st>>>(parts, grid, m, m_pad, G, Gf);
    return cudaGetLastError();
}

bool grouped_encode_gram_maps(const GInst& g, GMaps& out) {
    const bool ok_x = g.xf32 ? encode_2d(&out.xp, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, g.XP, g.d, g.n, g.ldp * 4, 32, 128,
                                         CU_TENSOR_MAP_SWIZZLE_128B)
                             : encode_bf16_2d(&out.xp, g.XP, g.d, g.n, g.ldp * 2, 64, 128);
    return ok_x && encode_bf16_2d(&out.q3, g.Q3, g.d, 3ull * g.m_pad, g.ldv * 2, 64, g.m_pad) &&
           encode_bf16_2d(&out.y3, g.Y3, g.ldy, 3ull * g.m_pad, g.ldy * 2, 64, g.m_pad);
}

// Split precision throughout (Algorithm 1, step 3 at the accuracy of the
// single-problem ACCURATE path): FP32 X in three pieces or BF16 X against three
// Q pieces, the leading product folded every 12 K-stages.
cudaError_t grouped_projected_gram(const GInst* gi, const GMaps* maps, GTable ygen32, GTable ygen16, GTable gram_items,
                                   GTable reduce_blocks, int max_m, int* status, int num_sms, cudaStream_t st) {
    const int m_pad_max = (int)rup(max_m, 32);
    cudaError_t e = cudaSuccess;
    if (ygen32.total > 0)
        e = launch_ygen<3, 3, true>(YgenGroup{gi, maps, ygen32}, ygen32.total, 12, m_pad_max, status, num_sms, st);
    if (e == cudaSuccess && ygen16.total > 0)
        e = launch_ygen<1, 3, false>(YgenGroup{gi, maps, ygen16}, ygen16.total, 12, m_pad_max, status, num_sms, st);
    if (e == cudaSuccess) e = launch_gram_y(GramGroup{gi, maps, gram_items}, gram_items.total, status, st);
    if (e != cudaSuccess) return e;
    note_launch();
    gram_parts_reduce_grouped_kernel<<<reduce_blocks.total, 256, 0, st>>>(gi, reduce_blocks);
    return cudaGetLastError();
}

cudaError_t pass_gram_set_wait_limit(uint64_t ns) { return tc::set_wait_limit(ns); }

}  // namespace ppca
