// Learned coarse-grid closure: a 1D convolutional network (5 layers, kernel 5,
// 64 hidden channels, ReLU) that maps coarse-grid moment fields to a
// correction of those fields.  Training and inference run in this file's
// kernels: BF16 weights and activations, FP32 accumulation on the tensor cores
// (tcgen05.mma with TMEM accumulators for the forward and backward-data
// convolutions, mma.sync m16n8k16 for the weight gradients), FP32 master
// weights updated by Adam.
//
// Layout: activations are channels-last, act[b][x][c] (bf16), with channel
// counts padded to multiples of 16; padded channels
// hold zeros and their weights stay zero.  Weights of layer l are
// W[co][j][ci] (tap j = 0..4 reads position x + j - 2).  Sample b is padded
// periodically (periodic[b] != 0) or by replicating its end values.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/qlbm.h"

namespace {

constexpr int kTaps = 5;
constexpr int kTM = 64;  // positions per CTA tile
// Resident weight-gradient CTAs per SM the kernel is compiled for.
#ifndef QL_WGRAD_MINBLOCKS
#define QL_WGRAD_MINBLOCKS 2
#endif
typedef __nv_bfloat16 bf16;

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// ldmatrix: lanes 8i..8i+7 give the 16-byte row addresses of 8x8 matrix i; each
// lane receives, per matrix, the element pair (row lane/4, columns 2 (lane%4),
// +1) of the matrix, or of its transpose with .trans (the mma.sync fragment
// layouts).
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const bf16 *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_trans(uint32_t (&r)[4], const bf16 *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x2_trans(uint32_t (&r)[2], const bf16 *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
                 : "=r"(r[0]), "=r"(r[1])
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma16816(float *d, const uint32_t *a, const uint32_t *b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Padding of a position outside [0, X): periodic image, copy of the nearest end
// value, or zero (the transposed convolution of the backward pass).
enum { PAD_ZERO = 0, PAD_PERIODIC = 1, PAD_REPLICATE = 2 };
// 16-byte asynchronous copy global -> shared; src_bytes 0 writes zeros and
// reads nothing.  Completion per thread by commit / wait groups.
__device__ __forceinline__ void cp_async16_zfill(void *smem_dst, const void *src, unsigned src_bytes)
{
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ int wrap_pos(int p, int X, int mode, bool *inside)
{
    *inside = true;
    if (p >= 0 && p < X) return p;
    if (mode == PAD_PERIODIC) return ((p % X) + X) % X;
    if (mode == PAD_REPLICATE) return p < 0 ? 0 : X - 1;
    *inside = false;
    return 0;
}

// ---------------------------------------------------------------------------
// Blackwell tensor cores (tcgen05): the A and B operands are read from shared
// memory through 64-bit matrix descriptors, the FP32 accumulator lives in
// tensor memory (TMEM) and is read back by tcgen05.ld.
//
// Shared-memory matrix descriptor, no swizzle, K-major canonical layout: core
// matrices of 8 rows x 16 bytes stored as 128 contiguous bytes; lbo is the byte
// distance between core matrices adjacent along K, sbo along M (or N).  Fields:
// address >> 4 in bits 0-13, lbo >> 4 in 16-29, sbo >> 4 in 32-45, descriptor
// version 1 in bits 46-47, base offset 0, layout type 0 (no swizzle) in 61-63.
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return uint64_t((addr >> 4) & 0x3FFF) | (uint64_t((lbo >> 4) & 0x3FFF) << 16) |
           (uint64_t((sbo >> 4) & 0x3FFF) << 32) | (uint64_t(1) << 46);
}
// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator (bits 4-5 =
// 1), BF16 A and B (bits 7-9 and 10-12 = 1), both K-major, N >> 3 in bits 17-22,
// M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}
__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, int accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
                 "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
                 : "memory");
}
__device__ __forceinline__ void mbar_init1(uint64_t *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// 16 consecutive FP32 columns of this thread's TMEM lane (lane = 32 (warp % 4) + lane id).
__device__ __forceinline__ void tmem_ld16(float (&v)[16], uint32_t taddr)
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}
// Polls of the tensor cores' completion barrier before a CTA gives up (bit 1 of
// the closure's error word; each try_wait may suspend the thread for a while).
constexpr uint32_t kMmaPolls = 1u << 20;

// Epilogues of the convolution kernel.
enum { EPI_RELU_BF16 = 0, EPI_F32 = 1, EPI_MASK_BF16 = 2 };

// Positions per tile of the convolution (the M of one tensor-core instruction).
constexpr int kConvM = 128;

// y[b][x][co] = sum_{j, ci} w[co][j][ci] in[b][x + j - 2][ci] (+ bias), then
//   EPI_RELU_BF16: relu, stored bf16;  EPI_F32: stored f32;
//   EPI_MASK_BF16: the transposed convolution of the backward pass: input
//     positions outside the sample are zero; at the two end positions of a
//     replicate-padded sample edge[b][side][co] is added (edge_grad_kernel);
//     then times (mask[b][x][co] > 0), stored bf16 (ReLU backward).
// An implicit GEMM per (sample, 128-position tile): M = positions, N = COUT,
// K = 5 CIN, on tcgen05.mma (M 128, N COUT, K 16 per instruction, issued by one
// thread) with the FP32 accumulator in TMEM.  Both operands are K-major in the
// no-swizzle canonical layout.  The input window of 132 positions is stored as
// [chunk of 8 channels][position][8], so every 8 consecutive positions of a
// chunk are one core matrix and tap j is the same descriptor moved by j rows
// (16 bytes): A(j) = window rows j .. j + 127.  The weights are stored as
// [K chunk = (j, 8 channels)][co][8].  Persistent CTAs load the layer's
// weights once, then walk the items with a grid stride, the next item's window
// copied in by cp.async while the tensor cores work on the current one; after
// each item's products complete (tcgen05.commit on an mbarrier), thread
// 32 w + l reads position 32 w + l of the tile (TMEM lane) and applies the
// epilogue.  A wait on the products that gives up sets bit 1 of *err.
template <int CIN, int COUT, int EPI>
__global__ void __launch_bounds__(128) conv_kernel(const bf16 *__restrict__ in, const bf16 *__restrict__ w,
                                                   const float *__restrict__ bias, const int *__restrict__ periodic,
                                                   int X, int B, void *__restrict__ out, const bf16 *__restrict__ mask,
                                                   const float *__restrict__ edge, unsigned *__restrict__ err)
{
    static_assert(CIN % 16 == 0 && COUT % 16 == 0 && COUT <= 256, "padded channels, one tcgen05 N");
    constexpr int KC = CIN / 8;                       // 8-channel chunks of a position
    constexpr int ROWS = kConvM + kTaps - 1;          // window positions
    constexpr int WCH = kTaps * KC;                   // weight chunks along K
    constexpr uint32_t ALBO = ROWS * 16, BLBO = COUT * 16;
    constexpr uint32_t NCOL = COUT < 32 ? 32 : COUT;  // TMEM columns (a power of 2, at least 32)
    constexpr int kWin = KC * ROWS * 8;               // bf16 per window stage
    extern __shared__ __align__(128) unsigned char smem[];
    bf16 *const ws = reinterpret_cast<bf16 *>(smem);  // [WCH][COUT][8]
    bf16 *const win_base = ws + WCH * COUT * 8;       // two stages of [KC][ROWS][8]
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t s_taddr;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    // W[co][j][ci] -> chunk r = j KC + ci / 8, row co
    for (int e = t; e < COUT * WCH; e += blockDim.x) {
        const int co = e / WCH, r = e % WCH;
        *reinterpret_cast<uint4 *>(ws + (r * COUT + co) * 8) =
            *reinterpret_cast<const uint4 *>(w + (size_t(co) * WCH + r) * 8);
    }
    if (t == 0) mbar_init1(&mbar);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_taddr)),
                     "r"(NCOL)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = s_taddr;
    const int tiles = (X + kConvM - 1) / kConvM;
    // cp.async of the input window of `item` into stage `st` (positions beyond the
    // padding are zero-filled: source size 0, nothing is read)
    auto stage_win = [&](int item, int st) {
        bf16 *win = win_base + st * kWin;
        const int b = item / tiles, x0 = (item % tiles) * kConvM;
        const int mode = periodic[b] != 0 ? PAD_PERIODIC : (EPI == EPI_MASK_BF16 ? PAD_ZERO : PAD_REPLICATE);
        for (int e = t; e < ROWS * KC; e += blockDim.x) {
            const int p = e / KC, c = e % KC;
            bool inside;
            const int x = wrap_pos(x0 - 2 + p, X, mode, &inside);
            const bf16 *src = inside ? in + (size_t(b) * X + x) * CIN + c * 8 : in;
            cp_async16_zfill(win + (c * ROWS + p) * 8, src, inside ? 16u : 0u);
        }
        cp_async_commit();
    };
    int st = 0;
    uint32_t phase = 0;
    bool failed = false;
    if (blockIdx.x < B * tiles) stage_win(blockIdx.x, 0);
    for (int item = blockIdx.x; item < B * tiles; item += gridDim.x, st ^= 1) {
        const int b = item / tiles, x0 = (item % tiles) * kConvM;
        const bool more = item + int(gridDim.x) < B * tiles;
        if (more) stage_win(item + gridDim.x, st ^ 1);
        if (more) cp_async_wait<1>();
        else cp_async_wait<0>();
        // this thread's copies (and, the first time, its weight stores) before the
        // tensor cores read them through the async proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t wa = smem_u32(win_base + st * kWin), wb = smem_u32(ws);
            int step = 0;
#pragma unroll
            for (int j = 0; j < kTaps; ++j)
#pragma unroll
                for (int kc = 0; kc < KC; kc += 2, ++step)
                    umma_bf16(taddr, umma_desc(wa + kc * ALBO + j * 16, ALBO, 128),
                              umma_desc(wb + (j * KC + kc) * BLBO, BLBO, 128), umma_idesc_bf16(kConvM, COUT), step);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&mbar))
                         : "memory");
        }
        // the thread's position and, for the backward pass, its ReLU mask (loaded
        // while the tensor cores work)
        const int m = warp * 32 + lane, x = x0 + m;
        const bool valid = x < X;
        uint4 mk[EPI == EPI_MASK_BF16 ? COUT / 8 : 1];
        if constexpr (EPI == EPI_MASK_BF16) {
#pragma unroll
            for (int v = 0; v < COUT / 8; ++v)
                mk[v] = valid ? *reinterpret_cast<const uint4 *>(mask + (size_t(b) * X + x) * COUT + v * 8)
                              : make_uint4(0u, 0u, 0u, 0u);
        }
        uint32_t polls = 0;
        while (!mbar_test(&mbar, phase) && ++polls < kMmaPolls) {
        }
        if (__syncthreads_or(polls >= kMmaPolls)) {
            if (t == 0) atomicOr(err, 2u);
            failed = true;
            break;
        }
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const bool per = periodic[b] != 0;
        const size_t o = (size_t(b) * X + (valid ? x : 0)) * COUT;
#pragma unroll
        for (int c0 = 0; c0 < COUT; c0 += 16) {
            float v[16];
            tmem_ld16(v, taddr + (uint32_t(warp * 32) << 16) + c0);
            if (!valid) continue;
            if (EPI != EPI_MASK_BF16) {
#pragma unroll
                for (int q = 0; q < 16; q += 4) {
                    const float4 bb = *reinterpret_cast<const float4 *>(bias + c0 + q);
                    v[q] += bb.x;
                    v[q + 1] += bb.y;
                    v[q + 2] += bb.z;
                    v[q + 3] += bb.w;
                }
            }
            if (EPI == EPI_F32) {
                float4 *dst = reinterpret_cast<float4 *>(static_cast<float *>(out) + o + c0);
#pragma unroll
                for (int q = 0; q < 4; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                continue;
            }
            if (EPI == EPI_MASK_BF16) {
                if (!per && (x == 0 || x == X - 1)) {
                    const float *eg = edge + (size_t(b) * 2 + (x != 0)) * COUT + c0;
#pragma unroll
                    for (int q = 0; q < 16; ++q) v[q] += eg[q];
                }
                const __nv_bfloat162 *mp = reinterpret_cast<const __nv_bfloat162 *>(&mk[c0 / 8]);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const __nv_bfloat162 mv = mp[q];
                    v[2 * q] = __bfloat162float(mv.x) > 0.f ? v[2 * q] : 0.f;
                    v[2 * q + 1] = __bfloat162float(mv.y) > 0.f ? v[2 * q + 1] : 0.f;
                }
            } else {
#pragma unroll
                for (int q = 0; q < 16; ++q) v[q] = fmaxf(v[q], 0.f);
            }
            uint4 pk[2];
            __nv_bfloat162 *pp = reinterpret_cast<__nv_bfloat162 *>(pk);
#pragma unroll
            for (int q = 0; q < 8; ++q) pp[q] = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
            uint4 *dst = reinterpret_cast<uint4 *>(static_cast<bf16 *>(out) + o + c0);
            dst[0] = pk[0];
            dst[1] = pk[1];
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();  // TMEM and this window stage are reused by later items
    }
    cp_async_wait<0>();
    if (failed) {  // let products still in flight land before their TMEM is freed
        uint32_t polls = 0;
        while (!mbar_test(&mbar, phase) && ++polls < kMmaPolls) {
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(NCOL) : "memory");
}

// Weight and bias gradients of one layer:
//   dW[co][j][ci] = sum_{b,x} dz[b][x][co] in[b][x + j - 2][ci],  db[co] = sum dz[b][x][co],
// a GEMM with M = COUT, N = 5 CIN, K = positions.  Each CTA accumulates over
// its share of the (sample, tile) items and writes a partial;
// reduce_partials_kernel sums the partials in a fixed order.  The dz tile and
// the input window are staged channels-last by 16-byte cp.async copies, two
// items deep; the transposed operands (K = positions contiguous) come from
// ldmatrix .trans.
// 8 warps: warp (mw, nw) holds couts [16 mw, 16 mw + 16) and NTW of the N/8
// column tiles.
template <int CIN, int COUT>
__global__ void __launch_bounds__(256, QL_WGRAD_MINBLOCKS) wgrad_kernel(const bf16 *__restrict__ dz, const bf16 *__restrict__ in,
                                                    const int *__restrict__ periodic, int X, int ntiles,
                                                    float *__restrict__ partial)
{
    static_assert(CIN % 8 == 0 && COUT % 16 == 0, "padded channels");
    constexpr int N = kTaps * CIN;
    constexpr int MT = COUT / 16;            // m tiles
    constexpr int NT = N / 8;                // n tiles
    constexpr int NW = 8 / MT;               // warps along N
    constexpr int NTW = (NT + NW - 1) / NW;  // n tiles per warp
    constexpr int DS = COUT + 8, IS = CIN + 8;  // smem row strides (bf16)
    extern __shared__ __align__(16) unsigned char smem[];
    // two stages of [kTM][DS] dz tile (positions x couts) and [kTM + 4][IS]
    // input window (positions x cins): the next item is copied in while the
    // current one is multiplied
    constexpr int kStage = kTM * DS + (kTM + 4) * IS;
    bf16 *const stage_base = reinterpret_cast<bf16 *>(smem);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, g = lane >> 2, tg = lane & 3;
    const int t8 = lane & 7, mat = lane >> 3;
    const int mw = warp % MT, nw = warp / MT;
    float acc[NTW][4];
#pragma unroll
    for (int n = 0; n < NTW; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
    float db = 0.f;
    const int tiles = (X + kTM - 1) / kTM;
    // cp.async of item `item` into stage `st`: positions outside the sample (and
    // outside the padding) are zero-filled (source size 0, nothing is read)
    auto stage_item = [&](int item, int st) {
        bf16 *sdz = stage_base + st * kStage, *sin = sdz + kTM * DS;
        const int b = item / tiles, x0 = (item % tiles) * kTM;
        const int mode = periodic[b] != 0 ? PAD_PERIODIC : PAD_REPLICATE;
        for (int e = t; e < kTM * (COUT / 8); e += blockDim.x) {
            const int p = e / (COUT / 8), v = e % (COUT / 8);
            const int x = x0 + p;
            const bf16 *src = x < X ? dz + (size_t(b) * X + x) * COUT + v * 8 : dz;
            cp_async16_zfill(sdz + p * DS + v * 8, src, x < X ? 16u : 0u);
        }
        for (int e = t; e < (kTM + 4) * (CIN / 8); e += blockDim.x) {
            const int p = e / (CIN / 8), v = e % (CIN / 8);
            bool inside;
            const int x = wrap_pos(x0 - 2 + p, X, mode, &inside);
            const bf16 *src = inside ? in + (size_t(b) * X + x) * CIN + v * 8 : in;
            cp_async16_zfill(sin + p * IS + v * 8, src, inside ? 16u : 0u);
        }
        cp_async_commit();
    };
    int st = 0;
    if (blockIdx.x < ntiles) stage_item(blockIdx.x, 0);
    for (int item = blockIdx.x; item < ntiles; item += gridDim.x, st ^= 1) {
        const bool more = item + int(gridDim.x) < ntiles;
        if (more) stage_item(item + gridDim.x, st ^ 1);
        if (more) cp_async_wait<1>();
        else cp_async_wait<0>();
        __syncthreads();
        const bf16 *sdz = stage_base + st * kStage, *sin = sdz + kTM * DS;
        // bias gradient: thread t < COUT sums column t of the dz tile
        if (t < COUT) {
            float s = 0.f;
            for (int p = 0; p < kTM; ++p) s += __bfloat162float(sdz[p * DS + t]);
            db += s;
        }
#pragma unroll
        for (int k0 = 0; k0 < kTM; k0 += 16) {
            // A[m = co][k = position] = sdz[k0 + k][16 mw + m]: transposed 8x8 blocks
            // (co 0-7 | 8-15) x (positions 0-7 | 8-15)
            uint32_t a[4];
            ldsm_x4_trans(a, sdz + (k0 + (mat >> 1) * 8 + t8) * DS + 16 * mw + (mat & 1) * 8);
#pragma unroll
            for (int n = 0; n < NTW; ++n) {
                const int nt = nw * NTW + n;
                if (nt >= NT) break;
                // column tile nt: tap j, cins [ci0, ci0 + 8); B[k][c] = in[x0 + k0 + k + j - 2][ci0 + c]
                // = sin[k0 + k + j][ci0 + c]: transposed blocks for k 0-7 and 8-15 (lanes 0-15)
                const int j = (nt * 8) / CIN, ci0 = (nt * 8) % CIN;
                uint32_t bb[2];
                ldsm_x2_trans(bb, sin + (k0 + (mat & 1) * 8 + t8 + j) * IS + ci0);
                mma16816(acc[n], a, bb);
            }
        }
        __syncthreads();  // this stage is refilled two items later
    }
    // partial[cta][co][col] with col = j CIN + ci, then the bias partials
    float *P = partial + size_t(blockIdx.x) * (COUT * N + COUT);
#pragma unroll
    for (int n = 0; n < NTW; ++n) {
        const int nt = nw * NTW + n;
        if (nt >= NT) break;
        const int col = nt * 8 + 2 * tg;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int co = 16 * mw + g + 8 * h;
            P[co * N + col] = acc[n][2 * h];
            P[co * N + col + 1] = acc[n][2 * h + 1];
        }
    }
    if (t < COUT) P[COUT * N + t] = db;
}

// Replicate padding feeds the end values a[0] and a[X-1] of a sample into the
// taps that reach past its ends, so their gradients get terms the zero-padded
// transposed convolution lacks:
//   left  (x = 0):     sum_co (W0 + W1)[co][ci] dz[0][co] + W0[co][ci] dz[1][co]
//   right (x = X - 1): sum_co (W3 + W4)[co][ci] dz[X-1][co] + W4[co][ci] dz[X-2][co]
// w is the forward layer's W[co][j][ci].  One block per side, kEdgeSamples
// samples and kEdgeChannels input channels: the two weight combinations of
// that side and channel range (the same for every sample) and the samples' end
// gradients are staged in shared memory once.
constexpr int kEdgeSamples = 16, kEdgeChannels = 16;
__global__ void __launch_bounds__(256) edge_grad_kernel(const bf16 *__restrict__ dz, const bf16 *__restrict__ w,
                                                        const int *__restrict__ periodic, int B, int X, int cout,
                                                        int cin, float *__restrict__ edge)
{
    __shared__ float s_a[64][kEdgeChannels], s_n[64][kEdgeChannels];  // [co][ci - c0], cout <= 64
    __shared__ float s_d0[kEdgeSamples][64], s_d1[kEdgeSamples][64];
    const int side = blockIdx.y, b0 = blockIdx.x * kEdgeSamples, c0 = blockIdx.z * kEdgeChannels, t = threadIdx.x;
    const int ja = side ? 3 : 0, jb = side ? 4 : 1, jn = side ? 4 : 0;
    for (int e = t; e < cout * kEdgeChannels; e += blockDim.x) {
        const int co = e / kEdgeChannels, cc = e - co * kEdgeChannels, ci = c0 + cc;
        float a = 0.f, n = 0.f;
        if (ci < cin) {
            a = __bfloat162float(w[(co * kTaps + ja) * cin + ci]) + __bfloat162float(w[(co * kTaps + jb) * cin + ci]);
            n = __bfloat162float(w[(co * kTaps + jn) * cin + ci]);
        }
        s_a[co][cc] = a;
        s_n[co][cc] = n;
    }
    for (int e = t; e < kEdgeSamples * cout; e += blockDim.x) {
        const int sm = e / cout, co = e - sm * cout, b = b0 + sm;
        float d0 = 0.f, d1 = 0.f;
        if (b < B) {
            d0 = __bfloat162float(dz[(size_t(b) * X + (side ? X - 1 : 0)) * cout + co]);
            d1 = __bfloat162float(dz[(size_t(b) * X + (side ? X - 2 : 1)) * cout + co]);
        }
        s_d0[sm][co] = d0;
        s_d1[sm][co] = d1;
    }
    __syncthreads();
    const int sm = t / kEdgeChannels, cc = t - sm * kEdgeChannels, b = b0 + sm, ci = c0 + cc;
    if (sm < kEdgeSamples && b < B && ci < cin) {
        float acc = 0.f;
        if (periodic[b] == 0)
            for (int co = 0; co < cout; ++co) {
                acc = fmaf(s_a[co][cc], s_d0[sm][co], acc);
                acc = fmaf(s_n[co][cc], s_d1[sm][co], acc);
            }
        edge[(size_t(b) * 2 + side) * cin + ci] = acc;
    }
}

// out[i] = sum_c partial[c][i] in a fixed order.  A block of 16 warps takes 128
// consecutive i (four per lane, 16-byte loads); warp w sums the parts c = w,
// w + 16, ... in four interleaved running sums (independent loads in flight),
// and the warp sums are added in warp order, so the result does not depend on
// scheduling.  len is a multiple of 4.
constexpr int kReduceWarps = 16;
__device__ __forceinline__ float4 add4(float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }
__global__ void __launch_bounds__(32 * kReduceWarps) reduce_partials_kernel(const float *__restrict__ partial,
                                                                           int nparts, int len,
                                                                           float *__restrict__ out)
{
    __shared__ float4 s_w[kReduceWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i4 = blockIdx.x * 32 + lane;  // float4 index
    const bool ok = 4 * i4 < len;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 s[4] = {z, z, z, z};
    if (ok) {
        const float4 *p = reinterpret_cast<const float4 *>(partial) + i4;
        const size_t row = size_t(len) / 4;
        int c = warp;
        for (; c + 3 * kReduceWarps < nparts; c += 4 * kReduceWarps)
#pragma unroll
            for (int r = 0; r < 4; ++r) s[r] = add4(s[r], p[size_t(c + r * kReduceWarps) * row]);
        for (int r = 0; c < nparts; c += kReduceWarps, ++r) s[r] = add4(s[r], p[size_t(c) * row]);
    }
    s_w[warp][lane] = add4(add4(s[0], s[1]), add4(s[2], s[3]));
    __syncthreads();
    if (warp == 0 && ok) {
        float4 r = s_w[0][lane];
        for (int k = 1; k < kReduceWarps; ++k) r = add4(r, s_w[k][lane]);
        reinterpret_cast<float4 *>(out)[i4] = r;
    }
}

// Input features (f32 [B][X][cin_real]) -> normalised bf16 [B][X][CINP].
__global__ void pack_input_kernel(const float *__restrict__ x, int64_t n, int cin, int cinp,
                                  const float *__restrict__ shift, const float *__restrict__ inv_scale,
                                  bf16 *__restrict__ out)
{
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= n * cinp) return;
    const int64_t pos = e / cinp;
    const int c = int(e % cinp);
    float v = 0.f;
    if (c < cin) v = (x[pos * cin + c] - shift[c]) * inv_scale[c];
    out[e] = __float2bfloat16(v);
}

// The same for the mini-batch idx[0..B) = perm[step B ..] (step read from the
// device) of a data set of n samples (X positions each), with the samples'
// padding kinds gathered into perb.  An index outside
// [0, n) sets *bad and reads sample 0 instead, so nothing is read out of bounds.
__global__ void pack_gather_kernel(const float *__restrict__ x, const int32_t *__restrict__ per,
                                   const int32_t *__restrict__ perm, const int *__restrict__ step, int64_t n, int B,
                                   int X, int cin, int cinp, const float *__restrict__ shift,
                                   const float *__restrict__ inv_scale, bf16 *__restrict__ out,
                                   int32_t *__restrict__ perb, unsigned *__restrict__ bad)
{
    const int32_t *__restrict__ idx = perm + int64_t(*step) * B;  // this step's samples
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e < B) {
        const int64_t k = idx[e];
        const bool ok = k >= 0 && k < n;
        if (!ok) atomicOr(bad, 1u);
        perb[e] = per[ok ? k : 0];
    }
    if (e >= int64_t(B) * X * cinp) return;
    const int64_t pos = e / cinp;
    const int c = int(e % cinp);
    const int64_t b = pos / X;
    int64_t k = idx[b];
    if (k < 0 || k >= n) k = 0;
    float v = 0.f;
    if (c < cin) v = (x[(k * X + (pos - b * X)) * cin + c] - shift[c]) * inv_scale[c];
    out[e] = __float2bfloat16(v);
}

// Mean squared error between prediction (f32 [B][X][COUTP], first cout used) and
// target / out_scale; writes dL/dpred (bf16, padded channels zero) and
// per-block partial sums of the squared error.
// y rows of the batch: y[b] directly, or y[idx[b]] of the whole data set
// (idx already checked by pack_gather_kernel; X positions per sample).
__global__ void mse_kernel(const float *__restrict__ pred, const float *__restrict__ y, const int32_t *__restrict__ idx,
                           const int *__restrict__ step, int X, int64_t npos, int cout, int coutp,
                           const float *__restrict__ inv_out_scale, float grad_scale, bf16 *__restrict__ dpred,
                           float *__restrict__ partial)
{
    // step (device, may be null): the batch is idx[step * B ..] of a training run's permutation
    if (idx && step) idx += int64_t(*step) * (npos / X);
    __shared__ float red[256];
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    float se = 0.f;
    if (e < npos * coutp) {
        const int64_t pos = e / coutp;
        const int c = int(e % coutp);
        float d = 0.f;
        if (c < cout) {
            int64_t row = pos;
            if (idx) {
                const int64_t b = pos / X;
                row = int64_t(idx[b]) * X + (pos - b * X);
            }
            d = pred[e] - y[row * cout + c] * inv_out_scale[c];
            se = d * d;
        }
        dpred[e] = __float2bfloat16(grad_scale * d);
    }
    red[threadIdx.x] = se;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// Prediction in physical units: y[pos][c] = pred[pos][c] * out_scale[c], c < cout.
__global__ void unpack_output_kernel(const float *__restrict__ pred, int64_t npos, int cout, int coutp,
                                     const float *__restrict__ out_scale, float *__restrict__ y)
{
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= npos * cout) return;
    const int64_t pos = e / cout;
    const int c = int(e % cout);
    y[e] = pred[pos * coutp + c] * out_scale[c];
}

// Mean loss of one batch from the per-block partial sums of mse_kernel, summed
// in a fixed order by one block of 256 threads: each thread adds its strided
// share in FP32, the thread sums are combined in FP64.
__global__ void loss_sum_kernel(const float *__restrict__ partial, int nparts, float scale, float *__restrict__ out,
                                const int *__restrict__ step)
{
    if (step) out += *step;
    __shared__ double red[256];
    // four independent running sums per thread (loads in flight), combined in order
    float s4[4] = {0.f, 0.f, 0.f, 0.f};
    int i = threadIdx.x;
    for (; i + 3 * int(blockDim.x) < nparts; i += 4 * blockDim.x)
#pragma unroll
        for (int r = 0; r < 4; ++r) s4[r] += partial[i + r * blockDim.x];
    for (int r = 0; i < nparts; i += blockDim.x, ++r) s4[r] += partial[i];
    red[threadIdx.x] = double(s4[0]) + double(s4[1]) + double(s4[2]) + double(s4[3]);
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (int(threadIdx.x) < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = float(red[0] * double(scale));
}

// Advances the device step counter of a training run (last node of a step).
__global__ void step_inc_kernel(int *step) { *step += 1; }

// Adam on FP32 master parameters; refreshes the bf16 weight copies, the
// tap-flipped transposed copies used by the backward pass, and the f32 biases.
constexpr int kAdamLayers = 8;  // layers whose bf16 copies the Adam pass refreshes itself
struct AdamArgs {
    float *param, *m, *v;
    const float *grad;
    int64_t n;
    float lr, b1, b2, eps, c1, c2;  // c1 = 1/(1-b1^t), c2 = 1/(1-b2^t)
    // training runs: lr, c1, c2 of step *step from device arrays (null: the scalars above)
    const int *step;
    const float *lr_arr, *c1_arr, *c2_arr;
    // bf16 copies written in the same pass (nl = 0: none): layer l's W[co][j][ci]
    // at woff[l] (cout[l] x 5 x cin[l]) into w16 and, tap-flipped and
    // transposed, into wt16 at the same offset
    bf16 *w16, *wt16;
    int nl;
    int64_t woff[kAdamLayers];
    int cout[kAdamLayers], cin[kAdamLayers];
};
__global__ void adam_kernel(AdamArgs a)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const float g = a.grad[i];
    const float m = a.b1 * a.m[i] + (1.f - a.b1) * g;
    const float v = a.b2 * a.v[i] + (1.f - a.b2) * g * g;
    a.m[i] = m;
    a.v[i] = v;
    float lr = a.lr, c1 = a.c1, c2 = a.c2;
    if (a.step) {
        const int t = *a.step;
        lr = a.lr_arr[t];
        c1 = a.c1_arr[t];
        c2 = a.c2_arr[t];
    }
    const float p = a.param[i] - lr * (m * c1) / (sqrtf(v * c2) + a.eps);
    a.param[i] = p;
    for (int l = 0; l < a.nl; ++l) {
        const int64_t e = i - a.woff[l];
        const int ci_ = a.cin[l], cout_ = a.cout[l];
        if (e >= 0 && e < int64_t(cout_) * kTaps * ci_) {
            const int co = int(e / (kTaps * ci_)), j = int((e / ci_) % kTaps), ci = int(e % ci_);
            const bf16 b = __float2bfloat16(p);
            a.w16[i] = b;
            a.wt16[a.woff[l] + (int64_t(ci) * kTaps + (kTaps - 1 - j)) * cout_ + co] = b;
            break;
        }
    }
}

// bf16 copies of one layer's weights: w[co][j][ci] and wt[ci][4 - j][co].
__global__ void cast_weights_kernel(const float *__restrict__ wf, int cout, int cin, bf16 *__restrict__ w,
                                    bf16 *__restrict__ wt)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= cout * kTaps * cin) return;
    const int co = e / (kTaps * cin), j = (e / cin) % kTaps, ci = e % cin;
    const bf16 v = __float2bfloat16(wf[e]);
    w[e] = v;
    wt[(ci * kTaps + (kTaps - 1 - j)) * cout + co] = v;
}

// ---------------------------------------------------------------------------
struct Layer {
    int cin, cout;    // padded
    int cin_real, cout_real;
    int64_t woff, boff;  // offsets of W [cout][5][cin] and bias [cout] in the f32 parameter vector
};

// Persistent grid of the convolution: the CTAs an SM holds by shared memory,
// at most as many as its 512 TMEM columns give accumulators (each CTA allocates
// its columns for the whole launch).
template <int CIN, int COUT, int EPI>
cudaError_t conv_launch(const bf16 *in, const bf16 *w, const float *bias, const int *per, int B, int X, void *out,
                        const bf16 *mask, const float *edge, unsigned *err, cudaStream_t s)
{
    constexpr size_t smem = 16 * (size_t(kTaps) * (CIN / 8) * COUT + 2 * size_t(CIN / 8) * (kConvM + kTaps - 1));
    constexpr int ncol = COUT < 32 ? 32 : COUT;
    auto k = conv_kernel<CIN, COUT, EPI>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 128, smem);
    if (e != cudaSuccess) return e;
    per_sm = std::max(1, std::min(per_sm, 512 / ncol));
    const int items = B * ((X + kConvM - 1) / kConvM);
    const int grid = std::max(1, std::min(items, std::max(1, sms) * per_sm));
    k<<<grid, 128, smem, s>>>(in, w, bias, per, X, B, out, mask, edge, err);
    return cudaGetLastError();
}

cudaError_t conv_any(int cin, int cout, int epi, const bf16 *in, const bf16 *w, const float *bias, const int *per,
                     int B, int X, void *out, const bf16 *mask, const float *edge, unsigned *err, cudaStream_t s)
{
#define QC(CI, CO, EP)                                                                 \
    if (cin == CI && cout == CO && epi == EP)                                          \
        return conv_launch<CI, CO, EP>(in, w, bias, per, B, X, out, mask, edge, err, s);
    QC(16, 64, EPI_RELU_BF16)
    QC(64, 64, EPI_RELU_BF16)
    QC(64, 16, EPI_F32)
    QC(16, 64, EPI_MASK_BF16)
    QC(64, 64, EPI_MASK_BF16)
#undef QC
    return cudaErrorInvalidValue;
}

template <int CIN, int COUT>
cudaError_t wgrad_launch(const bf16 *dz, const bf16 *in, const int *per, int B, int X, int grid, float *partial,
                         cudaStream_t s)
{
    constexpr size_t smem = 2 * sizeof(bf16) * (kTM * (COUT + 8) + (kTM + 4) * (CIN + 8));
    auto k = wgrad_kernel<CIN, COUT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    const int ntiles = B * ((X + kTM - 1) / kTM);
    k<<<grid, 256, smem, s>>>(dz, in, per, X, ntiles, partial);
    return cudaGetLastError();
}

cudaError_t wgrad_any(int cin, int cout, const bf16 *dz, const bf16 *in, const int *per, int B, int X, int grid,
                      float *partial, cudaStream_t s)
{
    if (cin == 16 && cout == 64) return wgrad_launch<16, 64>(dz, in, per, B, X, grid, partial, s);
    if (cin == 64 && cout == 64) return wgrad_launch<64, 64>(dz, in, per, B, X, grid, partial, s);
    if (cin == 64 && cout == 16) return wgrad_launch<64, 16>(dz, in, per, B, X, grid, partial, s);
    return cudaErrorInvalidValue;
}

}  // namespace

// ---------------------------------------------------------------------------
struct ql_closure {
    ql_closure_desc d;
    int device = 0;
    cudaStream_t stream = nullptr;
    ql_alloc_fn alloc = nullptr;
    ql_free_fn free_fn = nullptr;
    void *alloc_user = nullptr;
    std::vector<Layer> layers;
    int64_t nparam = 0;
    float *param = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    bf16 *w16 = nullptr, *wt16 = nullptr;  // per layer at woff
    std::vector<bf16 *> act;  // act[0] input (bf16), act[l] output of layer l (l < L)
    float *pred = nullptr;    // last layer output f32 [B][X][16]
    std::vector<bf16 *> dz;   // dz[l]: gradient wrt pre-activation of layer l (1-based), stored bf16
    float *partial = nullptr;
    float *loss_partial = nullptr;
    float *edge = nullptr;  // [max_batch][2][64] end-position gradient terms of replicate padding
    float *norm = nullptr;  // in_shift[8], in_inv_scale[8], out_scale[8], inv_out_scale[8]
    // padding kinds of ql_closure_train_steps' mini-batch and its out-of-range index flag
    int32_t *perb = nullptr;
    unsigned *bad = nullptr;
    // ql_closure_train_steps: one step captured as a graph (keyed by its pointers and sizes) and replayed;
    // the device step counter and the per-step lr, 1/(1-b1^t), 1/(1-b2^t) tables it reads
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    const void *gkey[5] = {};
    int64_t gkey_n = 0, gkey_B = 0;
    int *d_step = nullptr;
    float *d_sched = nullptr;
    int64_t sched_cap = 0;
    int wgrid = 0;
    int64_t step = 0;
    std::string err;
};

static std::string g_closure_error;

static ql_status cfail(ql_closure *c, ql_status st, const std::string &m)
{
    if (c) c->err = m; else g_closure_error = m;
    return st;
}

static void *calloc_dev(ql_closure *c, size_t bytes)
{
    if (c->alloc) return c->alloc(bytes, c->alloc_user);
    void *p = nullptr;
    return cudaMalloc(&p, bytes) == cudaSuccess ? p : nullptr;
}

static void cfree_dev(ql_closure *c, void *p)
{
    if (!p) return;
    if (c->free_fn) c->free_fn(p, c->alloc_user);
    else cudaFree(p);
}

static void closure_release(ql_closure *c)
{
    for (void *p : {(void *)c->param, (void *)c->grad, (void *)c->m, (void *)c->v, (void *)c->w16, (void *)c->wt16,
                    (void *)c->pred, (void *)c->partial, (void *)c->loss_partial, (void *)c->edge,
                    (void *)c->norm, (void *)c->perb, (void *)c->bad, (void *)c->d_step, (void *)c->d_sched})
        cfree_dev(c, p);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (bf16 *p : c->act) cfree_dev(c, p);
    for (bf16 *p : c->dz) cfree_dev(c, p);
}

#define QC_CUDA(c, call)                                                                               \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return cfail(c, QL_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

static ql_status refresh_weights(ql_closure *c)
{
    for (const Layer &L : c->layers) {
        const int n = L.cout * kTaps * L.cin;
        cast_weights_kernel<<<(n + 255) / 256, 256, 0, c->stream>>>(c->param + L.woff, L.cout, L.cin, c->w16 + L.woff,
                                                                    c->wt16 + L.woff);
    }
    QC_CUDA(c, cudaGetLastError());
    return QL_OK;
}

// splitmix64, for seeded He-uniform initial weights
static uint64_t splitmix(uint64_t &s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Forward pass of B samples already packed in act[0]; leaves pred.
static ql_status forward(ql_closure *c, const int *per, int B)
{
    const int X = c->d.positions, nl = int(c->layers.size());
    for (int l = 0; l < nl; ++l) {
        const Layer &L = c->layers[l];
        const bool last = l == nl - 1;
        void *out = last ? static_cast<void *>(c->pred) : static_cast<void *>(c->act[l + 1]);
        QC_CUDA(c, conv_any(L.cin, L.cout, last ? EPI_F32 : EPI_RELU_BF16, c->act[l], c->w16 + L.woff,
                            c->param + L.boff, per, B, X, out, nullptr, nullptr, c->bad, c->stream));
    }
    return QL_OK;
}

static ql_status pack(ql_closure *c, const float *x, int B)
{
    const int64_t npos = int64_t(B) * c->d.positions;
    const int cinp = c->layers[0].cin;
    pack_input_kernel<<<unsigned((npos * cinp + 255) / 256), 256, 0, c->stream>>>(
        x, npos, c->d.in_channels, cinp, c->norm, c->norm + 8, c->act[0]);
    QC_CUDA(c, cudaGetLastError());
    return QL_OK;
}

static ql_status adam_step(ql_closure *c, float lr);

// The device flags (synchronises): bit 0, a mini-batch index outside the data
// set; bit 1, a convolution that gave up waiting for its tensor-core products.
static ql_status check_flags(ql_closure *c)
{
    unsigned bad = 0;
    QC_CUDA(c, cudaMemcpyAsync(&bad, c->bad, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    QC_CUDA(c, cudaStreamSynchronize(c->stream));
    if (bad & 2u) return cfail(c, QL_ECUDA, "a convolution gave up waiting for its tensor-core products");
    if (bad & 1u) return cfail(c, QL_EINVAL, "perm holds a sample index outside [0, n); sample 0 was used in its place");
    return QL_OK;
}

static ql_status enqueue_train_step(ql_closure *c, const float *x, const float *y, const int32_t *periodic,
                                    int64_t n, const int32_t *perm, int64_t B, float *losses);

// Loss, gradients of all parameters into c->grad; loss (host) if not null.
static ql_status backward(ql_closure *c, const float *y, const int32_t *yidx, const int *ystep, const int *per, int B,
                          float *loss)
{
    const int X = c->d.positions, nl = int(c->layers.size());
    const int64_t npos = int64_t(B) * X;
    const int coutp = c->layers[nl - 1].cout;
    const int64_t nel = npos * coutp;
    const unsigned nb = unsigned((nel + 255) / 256);
    const float gscale = 2.f / float(npos * c->d.out_channels);
    mse_kernel<<<nb, 256, 0, c->stream>>>(c->pred, y, yidx, ystep, X, npos, c->d.out_channels, coutp, c->norm + 24,
                                          gscale,
                                          c->dz[nl - 1], c->loss_partial);
    QC_CUDA(c, cudaGetLastError());
    for (int l = nl - 1; l >= 0; --l) {
        const Layer &L = c->layers[l];
        const int len = L.cout * kTaps * L.cin + L.cout;  // a multiple of 4 (channels are padded to 16)
        if (len % 4 != 0) return cfail(c, QL_EUNSUPPORTED, "channel padding");
        QC_CUDA(c, wgrad_any(L.cin, L.cout, c->dz[l], c->act[l], per, B, X, c->wgrid, c->partial, c->stream));
        // partial layout per CTA: [cout][5 cin] then [cout]; W and b are contiguous in the parameter vector
        reduce_partials_kernel<<<(len + 127) / 128, 32 * kReduceWarps, 0, c->stream>>>(c->partial, c->wgrid, len,
                                                                                     c->grad + L.woff);
        QC_CUDA(c, cudaGetLastError());
        if (l > 0) {
            // dz[l-1] = (W^T * dz[l] + end terms of replicate padding) masked by act[l] > 0
            // (act[l] is the output of layer l-1)
            static_assert(kEdgeSamples * kEdgeChannels == 256, "one output per thread");
            edge_grad_kernel<<<dim3((B + kEdgeSamples - 1) / kEdgeSamples, 2, (L.cin + kEdgeChannels - 1) / kEdgeChannels),
                               256, 0, c->stream>>>(
                c->dz[l], c->w16 + L.woff, per, B, X, L.cout, L.cin,
                                                                 c->edge);
            QC_CUDA(c, cudaGetLastError());
            QC_CUDA(c, conv_any(L.cout, L.cin, EPI_MASK_BF16, c->dz[l], c->wt16 + L.woff, nullptr, per, B, X,
                                c->dz[l - 1], c->act[l], c->edge, c->bad, c->stream));
        }
    }
    if (loss) {
        std::vector<float> h(nb);
        QC_CUDA(c, cudaMemcpyAsync(h.data(), c->loss_partial, sizeof(float) * nb, cudaMemcpyDeviceToHost, c->stream));
        QC_CUDA(c, cudaStreamSynchronize(c->stream));
        double s = 0;
        for (float v : h) s += v;
        *loss = float(s / double(npos * c->d.out_channels));
    }
    return QL_OK;
}

extern "C" {

ql_status ql_closure_create(const ql_closure_desc *d, const ql_opts *opts, ql_closure **out)
{
    if (out) *out = nullptr;
    if (!d || !opts || !out) return cfail(nullptr, QL_EINVAL, "null argument");
    if (d->ksize != kTaps || d->layers < 2 || d->width != 64 || d->in_channels < 1 || d->in_channels > 8 ||
        d->out_channels < 1 || d->out_channels > 8 || d->positions < 16 || d->max_batch < 1)
        return cfail(nullptr, QL_EUNSUPPORTED,
                     "supported: ksize 5, width 64, >= 2 layers, 1..8 inputs, 1..8 outputs, >= 16 positions");
    ql_closure *c = new ql_closure();
    c->d = *d;
    c->device = opts->device;
    c->alloc = opts->alloc;
    c->free_fn = opts->free;
    c->alloc_user = opts->alloc_user;
    c->stream = static_cast<cudaStream_t>(opts->stream);
    auto bail = [&](ql_status st, const std::string &m) {
        closure_release(c);
        delete c;
        return cfail(nullptr, st, m);
    };
    if (cudaSetDevice(c->device) != cudaSuccess) return bail(QL_ECUDA, "cudaSetDevice failed");
    int64_t off = 0;
    for (int l = 0; l < d->layers; ++l) {
        Layer L;
        L.cin_real = l == 0 ? d->in_channels : 64;
        L.cout_real = l == d->layers - 1 ? d->out_channels : 64;
        L.cin = l == 0 ? 16 : 64;
        L.cout = l == d->layers - 1 ? 16 : 64;
        L.woff = off;
        off += int64_t(L.cout) * kTaps * L.cin;
        L.boff = off;
        off += L.cout;
        c->layers.push_back(L);
    }
    c->nparam = off;
    const int X = d->positions, B = d->max_batch;
    const int64_t npos = int64_t(B) * X;
    c->param = static_cast<float *>(calloc_dev(c, sizeof(float) * off));
    c->grad = static_cast<float *>(calloc_dev(c, sizeof(float) * off));
    c->m = static_cast<float *>(calloc_dev(c, sizeof(float) * off));
    c->v = static_cast<float *>(calloc_dev(c, sizeof(float) * off));
    c->w16 = static_cast<bf16 *>(calloc_dev(c, sizeof(bf16) * off));
    c->wt16 = static_cast<bf16 *>(calloc_dev(c, sizeof(bf16) * off));
    c->pred = static_cast<float *>(calloc_dev(c, sizeof(float) * npos * 16));
    c->norm = static_cast<float *>(calloc_dev(c, sizeof(float) * 32));
    for (int l = 0; l < d->layers; ++l) {
        c->act.push_back(static_cast<bf16 *>(calloc_dev(c, sizeof(bf16) * npos * c->layers[l].cin)));
        c->dz.push_back(static_cast<bf16 *>(calloc_dev(c, sizeof(bf16) * npos * c->layers[l].cout)));
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    c->wgrid = sms > 0 ? 2 * sms : 256;
    c->partial = static_cast<float *>(calloc_dev(c, sizeof(float) * size_t(c->wgrid) * (64 * kTaps * 64 + 64)));
    c->loss_partial = static_cast<float *>(calloc_dev(c, sizeof(float) * ((npos * 16 + 255) / 256)));
    c->edge = static_cast<float *>(calloc_dev(c, sizeof(float) * size_t(B) * 2 * 64));
    c->perb = static_cast<int32_t *>(calloc_dev(c, sizeof(int32_t) * size_t(B)));
    c->bad = static_cast<unsigned *>(calloc_dev(c, sizeof(unsigned)));
    bool ok = c->param && c->grad && c->m && c->v && c->w16 && c->wt16 && c->pred && c->norm && c->partial &&
              c->loss_partial && c->edge && c->perb && c->bad;
    for (int l = 0; l < d->layers; ++l) ok = ok && c->act[l] && c->dz[l];
    if (!ok) return bail(QL_ENOMEM, "closure allocation failed");

    // seeded He-uniform weights (real channels only), zero biases and padding
    std::vector<float> h(off, 0.f);
    uint64_t s = d->seed;
    for (size_t l = 0; l < c->layers.size(); ++l) {
        const Layer &L = c->layers[l];
        const float a = sqrtf(6.f / float(kTaps * L.cin_real)) * (l + 1 == c->layers.size() ? 0.1f : 1.f);
        for (int co = 0; co < L.cout_real; ++co)
            for (int j = 0; j < kTaps; ++j)
                for (int ci = 0; ci < L.cin_real; ++ci) {
                    const double u = double(splitmix(s) >> 11) * (1.0 / 9007199254740992.0);
                    h[L.woff + (int64_t(co) * kTaps + j) * L.cin + ci] = float((2.0 * u - 1.0) * a);
                }
    }
    float nrm[32];
    for (int i = 0; i < 8; ++i) {
        nrm[i] = d->in_shift[i];
        nrm[8 + i] = d->in_scale[i] != 0.f ? 1.f / d->in_scale[i] : 1.f;
        nrm[16 + i] = d->out_scale[i] != 0.f ? d->out_scale[i] : 1.f;
        nrm[24 + i] = 1.f / nrm[16 + i];
    }
    cudaError_t e = cudaMemcpyAsync(c->param, h.data(), sizeof(float) * off, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->m, 0, sizeof(float) * off, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->v, 0, sizeof(float) * off, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->norm, nrm, sizeof(nrm), cudaMemcpyHostToDevice, c->stream);
    for (int l = 0; l < d->layers && e == cudaSuccess; ++l) {
        e = cudaMemsetAsync(c->act[l], 0, sizeof(bf16) * npos * c->layers[l].cin, c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->dz[l], 0, sizeof(bf16) * npos * c->layers[l].cout, c->stream);
    }
    if (e != cudaSuccess) return bail(QL_ECUDA, std::string("closure set-up: ") + cudaGetErrorString(e));
    if (refresh_weights(c) != QL_OK) return bail(QL_ECUDA, c->err);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return bail(QL_ECUDA, "closure set-up sync failed");
    *out = c;
    return QL_OK;
}

ql_status ql_closure_forward(ql_closure *c, const float *x, const int32_t *periodic, int64_t B, float *y)
{
    if (!c || !x || !periodic || !y || B < 1 || B > c->d.max_batch) return cfail(c, QL_EINVAL, "bad arguments");
    ql_status st = pack(c, x, int(B));
    if (st == QL_OK) st = forward(c, periodic, int(B));
    if (st != QL_OK) return st;
    const int64_t npos = B * c->d.positions;
    unpack_output_kernel<<<unsigned((npos * c->d.out_channels + 255) / 256), 256, 0, c->stream>>>(
        c->pred, npos, c->d.out_channels, c->layers.back().cout, c->norm + 16, y);
    QC_CUDA(c, cudaGetLastError());
    return QL_OK;
}

ql_status ql_closure_gradients(ql_closure *c, const float *x, const float *y, const int32_t *periodic, int64_t B,
                               float *loss, float *grad_host)
{
    if (!c || !x || !y || !periodic || B < 1 || B > c->d.max_batch) return cfail(c, QL_EINVAL, "bad arguments");
    ql_status st = pack(c, x, int(B));
    if (st == QL_OK) st = forward(c, periodic, int(B));
    if (st == QL_OK) st = backward(c, y, nullptr, nullptr, periodic, int(B), loss);
    if (st != QL_OK) return st;
    if (grad_host) {
        QC_CUDA(c, cudaMemcpyAsync(grad_host, c->grad, sizeof(float) * c->nparam, cudaMemcpyDeviceToHost, c->stream));
        QC_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return grad_host || loss ? check_flags(c) : QL_OK;
}

ql_status ql_closure_train_step(ql_closure *c, const float *x, const float *y, const int32_t *periodic, int64_t B,
                                float lr, float *loss)
{
    ql_status st = ql_closure_gradients(c, x, y, periodic, B, loss, nullptr);
    if (st != QL_OK) return st;
    return adam_step(c, lr);
}

ql_status ql_closure_train_steps(ql_closure *c, const float *x, const float *y, const int32_t *periodic, int64_t n,
                                 const int32_t *perm, int64_t nsteps, int64_t B, const float *lr, float *losses)
{
    if (!c || !x || !y || !periodic || !perm || n < 1 || nsteps < 0 || B < 1 || B > c->d.max_batch ||
        (nsteps > 0 && !lr))
        return cfail(c, QL_EINVAL, "bad arguments");
    QC_CUDA(c, cudaMemsetAsync(c->bad, 0, sizeof(unsigned), c->stream));
    if (nsteps > 0) {
        if (!c->d_step) {
            c->d_step = static_cast<int *>(calloc_dev(c, sizeof(int)));
            if (!c->d_step) return cfail(c, QL_ENOMEM, "step counter allocation failed");
        }
        if (nsteps > c->sched_cap) {
            cfree_dev(c, c->d_sched);
            c->sched_cap = 0;
            c->d_sched = static_cast<float *>(calloc_dev(c, sizeof(float) * 3 * size_t(nsteps)));
            if (!c->d_sched) return cfail(c, QL_ENOMEM, "schedule allocation failed");
            c->sched_cap = nsteps;
            if (c->gexec) cudaGraphExecDestroy(c->gexec);
            c->gexec = nullptr;
        }
        // the schedule of steps step+1 .. step+nsteps, in the arithmetic of the single-step path
        const int64_t cap = c->sched_cap;
        std::vector<float> h(size_t(3 * cap), 0.f);
        for (int64_t s = 0; s < nsteps; ++s) {
            const double t = double(c->step + s + 1);
            h[size_t(s)] = lr[s];
            h[size_t(cap + s)] = float(1.0 / (1.0 - pow(0.9, t)));
            h[size_t(2 * cap + s)] = float(1.0 / (1.0 - pow(0.999, t)));
        }
        QC_CUDA(c, cudaMemcpyAsync(c->d_sched, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice, c->stream));
        QC_CUDA(c, cudaMemsetAsync(c->d_step, 0, sizeof(int), c->stream));

        const void *key[5] = {x, y, periodic, perm, losses};
        if (c->gexec && (!std::equal(key, key + 5, c->gkey) || c->gkey_n != n || c->gkey_B != B)) {
            cudaGraphExecDestroy(c->gexec);
            c->gexec = nullptr;
        }
        if (!c->gexec) {
            // capture on a stream of our own (the caller's may be the legacy default stream)
            if (!c->cap_stream) QC_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
            cudaStream_t user = c->stream;
            c->stream = c->cap_stream;
            cudaGraph_t g = nullptr;
            ql_status st = QL_ECUDA;
            if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
                st = enqueue_train_step(c, x, y, periodic, n, perm, B, losses);
                if (cudaStreamEndCapture(c->stream, &g) != cudaSuccess) st = QL_ECUDA;
            }
            c->stream = user;
            if (st == QL_OK && cudaGraphInstantiate(&c->gexec, g, 0) != cudaSuccess) c->gexec = nullptr;
            if (g) cudaGraphDestroy(g);
            (void)cudaGetLastError();  // a capture that failed leaves the plain launches below
            std::copy(key, key + 5, c->gkey);
            c->gkey_n = n;
            c->gkey_B = B;
        }
        for (int64_t s = 0; s < nsteps; ++s) {
            if (c->gexec) {
                QC_CUDA(c, cudaGraphLaunch(c->gexec, c->stream));
            } else {
                ql_status st = enqueue_train_step(c, x, y, periodic, n, perm, B, losses);
                if (st != QL_OK) return st;
            }
        }
        c->step += nsteps;
    }
    return check_flags(c);
}

}  // extern "C"

static AdamArgs adam_args(ql_closure *c);

static ql_status adam_step(ql_closure *c, float lr)
{
    c->step += 1;
    AdamArgs a = adam_args(c);
    a.lr = lr;
    a.c1 = float(1.0 / (1.0 - pow(0.9, double(c->step))));
    a.c2 = float(1.0 / (1.0 - pow(0.999, double(c->step))));
    adam_kernel<<<unsigned((c->nparam + 255) / 256), 256, 0, c->stream>>>(a);
    QC_CUDA(c, cudaGetLastError());
    return a.nl ? QL_OK : refresh_weights(c);
}

static AdamArgs adam_args(ql_closure *c)
{
    AdamArgs a;
    a.param = c->param;
    a.m = c->m;
    a.v = c->v;
    a.grad = c->grad;
    a.n = c->nparam;
    a.lr = a.c1 = a.c2 = 0.f;
    a.b1 = 0.9f;
    a.b2 = 0.999f;
    a.eps = 1e-8f;
    a.step = nullptr;
    a.lr_arr = a.c1_arr = a.c2_arr = nullptr;
    const bool fused = c->layers.size() <= size_t(kAdamLayers);
    a.w16 = c->w16;
    a.wt16 = c->wt16;
    a.nl = fused ? int(c->layers.size()) : 0;
    for (int l = 0; l < a.nl; ++l) {
        a.woff[l] = c->layers[l].woff;
        a.cout[l] = c->layers[l].cout;
        a.cin[l] = c->layers[l].cin;
    }
    return a;
}

// One step of a training run on c->stream: the mini-batch perm[t B ..], the loss
// slot losses[t] (losses may be null) and the schedule entries are those of the
// device step counter t, which the last launch advances.
static ql_status enqueue_train_step(ql_closure *c, const float *x, const float *y, const int32_t *periodic,
                                    int64_t n, const int32_t *perm, int64_t B, float *losses)
{
    const int X = c->d.positions;
    const int64_t npos = B * X;
    const unsigned nb = unsigned((npos * c->layers.back().cout + 255) / 256);
    const float lscale = float(1.0 / double(npos * c->d.out_channels));
    const int cinp = c->layers[0].cin;
    pack_gather_kernel<<<unsigned((B * X * cinp + 255) / 256), 256, 0, c->stream>>>(
        x, periodic, perm, c->d_step, n, int(B), X, c->d.in_channels, cinp, c->norm, c->norm + 8, c->act[0], c->perb,
        c->bad);
    QC_CUDA(c, cudaGetLastError());
    ql_status st = forward(c, c->perb, int(B));
    if (st == QL_OK) st = backward(c, y, perm, c->d_step, c->perb, int(B), nullptr);
    if (st != QL_OK) return st;
    if (losses) {
        loss_sum_kernel<<<1, 256, 0, c->stream>>>(c->loss_partial, int(nb), lscale, losses, c->d_step);
        QC_CUDA(c, cudaGetLastError());
    }
    AdamArgs a = adam_args(c);
    a.step = c->d_step;
    a.lr_arr = c->d_sched;
    a.c1_arr = c->d_sched + c->sched_cap;
    a.c2_arr = c->d_sched + 2 * c->sched_cap;
    adam_kernel<<<unsigned((c->nparam + 255) / 256), 256, 0, c->stream>>>(a);
    QC_CUDA(c, cudaGetLastError());
    if (!a.nl) {
        st = refresh_weights(c);
        if (st != QL_OK) return st;
    }
    step_inc_kernel<<<1, 1, 0, c->stream>>>(c->d_step);
    QC_CUDA(c, cudaGetLastError());
    return QL_OK;
}

extern "C" {

ql_status ql_closure_params(ql_closure *c, float *get_host, const float *set_host, int64_t *count)
{
    if (!c) return cfail(c, QL_EINVAL, "null closure");
    if (count) *count = c->nparam;
    if (get_host) {
        QC_CUDA(c, cudaMemcpyAsync(get_host, c->param, sizeof(float) * c->nparam, cudaMemcpyDeviceToHost, c->stream));
        QC_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    if (set_host) {
        QC_CUDA(c, cudaMemcpyAsync(c->param, set_host, sizeof(float) * c->nparam, cudaMemcpyHostToDevice, c->stream));
        ql_status st = refresh_weights(c);
        if (st != QL_OK) return st;
        QC_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return QL_OK;
}

ql_status ql_closure_destroy(ql_closure *c)
{
    if (!c) return QL_OK;
    cudaStreamSynchronize(c->stream);
    closure_release(c);
    delete c;
    return QL_OK;
}

const char *ql_closure_last_error(const ql_closure *c) { return c ? c->err.c_str() : g_closure_error.c_str(); }

}  // extern "C"
