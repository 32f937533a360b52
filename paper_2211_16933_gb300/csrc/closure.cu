// Learned coarse-grid closure: a 1D convolutional network (5 layers, kernel 5,
// 64 hidden channels, ReLU) that maps coarse-grid moment fields to a
// correction of those fields.  Training and inference run in this file's
// kernels: BF16 weights and activations, FP32 accumulation on the tensor cores
// (tcgen05.mma with TMEM accumulators: the forward and backward-data
// convolutions and the weight gradients), FP32 master weights updated by Adam.
//
// Layout: activations and their gradients are bf16 [B][X][C] tensors stored
// chunk-major (16-byte rows of 8 channels, see cm_index), with channel counts
// padded to multiples of 16; padded channels hold zeros and their weights
// stay zero.  Weights of layer l are
// W[co][j][ci] (tap j = 0..4 reads position x + j - 2).  Sample b is padded
// periodically (periodic[b] != 0) or by replicating its end values.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <string>
#include <vector>

#include "../../include/qlbm.h"

namespace {

constexpr int kTaps = 5;
constexpr int kMaxDevices = 64;  // devices whose launch shapes are remembered
typedef __nv_bfloat16 bf16;

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// Padding of a position outside [0, X): periodic image, copy of the nearest end
// value, or zero (the transposed convolution of the backward pass).
enum { PAD_ZERO = 0, PAD_PERIODIC = 1, PAD_REPLICATE = 2 };
__device__ __forceinline__ int wrap_pos(int p, int X, int mode, bool *inside)
{
    *inside = true;
    if (p >= 0 && p < X) return p;
    if (mode == PAD_PERIODIC) return ((p % X) + X) % X;
    if (mode == PAD_REPLICATE) return p < 0 ? 0 : X - 1;
    *inside = false;
    return 0;
}

// Programmatic dependent launch: every kernel of the network is launched so that
// it may start while the kernel before it in the stream is finishing.  Each
// one calls pdl_wait() before it touches memory that kernel writes or reads
// (the wait returns once that kernel has completed and its writes are
// visible), and pdl_trigger() only after that, so that when a kernel starts,
// every kernel two or more places before it has completed.  Work that reads
// nothing a recent kernel writes (barrier set-up, tensor-memory allocation,
// the weight copy of a convolution, which only Adam writes, at the end of a
// step) goes before the wait and overlaps the previous kernel's tail.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

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
// 16 consecutive FP32 columns of this thread's TMEM lane (lane = 32 (warp % 4) +
// lane id), without waiting for them: tmem_wait() makes them usable.
__device__ __forceinline__ void tmem_ld16(uint32_t *r, uint32_t taddr)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
}
// Waits for this thread's tcgen05.ld; the registers pass through an empty asm
// after the wait, so no use of them is scheduled before it.
template <int N>
__device__ __forceinline__ void tmem_wait(uint32_t (&r)[N])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < N; ++q) asm volatile("" : "+r"(r[q])::"memory");
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// Polls of an mbarrier before a thread gives up (bit 1 of the closure's error
// word; each try_wait may suspend the thread for a while).
constexpr uint32_t kMmaPolls = 1u << 20;
// Waits until the phase of parity `parity` of *bar has completed.  Gives up
// (false) after kMmaPolls polls, or early once another role of the CTA has
// given up (*abort != 0; null: never early).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, const volatile int *abort)
{
    for (uint32_t polls = 0; !mbar_test(bar, parity);) {
        if (++polls >= kMmaPolls) return false;
        if (abort && (polls & 63u) == 0 && *abort) return false;
    }
    return true;
}
__device__ __forceinline__ void give_up(volatile int *abort, unsigned *err)
{
    *abort = 1;
    atomicOr(err, 2u);
}

// Chunk-major layout of the network's [B][X][C] tensors: the channels of a
// position are split into 16-byte rows of V elements (8 bf16 or 4 f32), and
// row q of sample b holds those V channels for every position in turn.
// Element (b, x, c) sits at ((b (C / V) + c / V) X + x) V + c % V.  A window
// of consecutive positions of one row is contiguous (one bulk copy), and a
// warp whose lanes take consecutive positions reads or writes 512 contiguous
// bytes per row.
__host__ __device__ __forceinline__ int64_t cm_index(int64_t b, int64_t x, int c, int C, int X, int V)
{
    return ((b * (C / V) + c / V) * X + x) * V + c % V;
}

// The bf16 weight copies of a layer (cout x 5 x cin) are stored in the order
// a convolution CTA stages them, so that one bulk copy brings them in: W[co][j][ci]
// at [K chunk r = j (cin / 8) + ci / 8][co][8].
__host__ __device__ __forceinline__ int64_t wstage_index(int co, int j, int ci, int cout, int cin)
{
    return (int64_t(j * (cin / 8) + ci / 8) * cout + co) * 8 + ci % 8;
}

// Bulk copy (TMA engine, no tensor map) of `bytes` global -> shared, counted
// against the transaction bytes of *bar; 16-byte aligned addresses, bytes a
// multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// Warp roles of the two tensor-core kernels: epilogue warps 0 .. E - 1 (warp w
// may access TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31), warp E copies the
// operands into shared memory, one thread of warp E + 1 issues the tensor-core
// instructions.
__host__ __device__ constexpr int role_threads(int epi_warps) { return 32 * (epi_warps + 2); }
// Epilogue warps of the convolution: two per TMEM lane quarter (each takes half
// the output channels) for 64 channels, one for fewer.
__host__ __device__ constexpr int conv_epi_warps(int cout) { return cout >= 64 ? 8 : 4; }
constexpr int kWgradEpiWarps = 4;
// Operand stages in shared memory.
constexpr int kConvStages = 4, kWgradStages = 4;

// Epilogues of the convolution kernel.
enum { EPI_RELU_BF16 = 0, EPI_F32 = 1, EPI_MASK_BF16 = 2 };

// Positions per tile of the convolution (the M of one tensor-core instruction).
constexpr int kConvM = 128;

// Fills stage rows 0 .. rows - 1 = positions x0 - halo .. of sample b of a
// chunk-major operand (C channels, [chunk][row][8] in shared memory) with the
// copy warp: lane 0 has the TMA engine copy the positions inside [0, X) of
// each chunk (one bulk copy per chunk), the lanes write the others (`mode`:
// zero, periodic image or nearest end value) with plain stores before it.
// Every lane then arrives on *full (32 arrivals; lane 0 also adds the bulk
// bytes to the phase's transaction count).
template <int C>
__device__ __forceinline__ void fill_rows(bf16 *dst, const bf16 *src, int b, int x0, int halo, int rows, int X,
                                          int mode, int lane, uint64_t *full)
{
    constexpr int KC = C / 8;
    const int first = x0 - halo;                                   // position of stage row 0
    const int lo = first < 0 ? 0 : first, hi = first + rows > X ? X : first + rows;  // inside [lo, hi)
    const int nl = lo - first, nr = first + rows - hi;            // rows before and after
    for (int e = lane; e < (nl + nr) * KC; e += 32) {
        const int r = e / KC, c = e % KC, p = r < nl ? r : (hi - first) + (r - nl);
        bool inside;
        const int x = wrap_pos(first + p, X, mode, &inside);
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (inside) v = *reinterpret_cast<const uint4 *>(src + cm_index(b, x, c * 8, C, X, 8));
        *reinterpret_cast<uint4 *>(dst + (c * rows + p) * 8) = v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // plain stores before the tensor cores' reads
    __syncwarp();
    if (lane == 0) {
        const uint32_t bytes = uint32_t(hi - lo) * 16u;
        mbar_arrive_tx(full, KC * bytes);
        for (int c = 0; c < KC; ++c)
            bulk_g2s(dst + (c * rows + nl) * 8, src + cm_index(b, lo, c * 8, C, X, 8), bytes, full);
    } else {
        mbar_arrive(full);
    }
}

// The copy warp before it leaves: the bulk copies of its last fills (items
// max(0, n - ns) .. n - 1 of stages full[item % ns]) have landed, so that none
// writes to shared memory after the CTA has ended, whatever the other roles did.
__device__ __forceinline__ void drain_fills(uint64_t *full, int ns, int n)
{
    for (int r = n - ns < 0 ? 0 : n - ns; r < n; ++r) mbar_wait(&full[r % ns], (r / ns) & 1, nullptr);
}

// y[b][x][co] = sum_{j, ci} w[co][j][ci] in[b][x + j - 2][ci] (+ bias), then
//   EPI_RELU_BF16: relu, stored bf16;  EPI_F32: stored f32;
//   EPI_MASK_BF16: the transposed convolution of the backward pass: input
//     positions outside the sample are zero; at the two end positions of a
//     replicate-padded sample edge[b][side][co] is added (edge_grad_kernel);
//     then times (mask[b][x][co] > 0), stored bf16 (ReLU backward).
// Tensors are chunk-major (cm_index; f32 output in rows of 4).
// An implicit GEMM per (sample, 128-position tile) item: M = positions, N =
// COUT, K = 5 CIN, on tcgen05.mma (M 128, N COUT, K 16 per instruction) with
// the FP32 accumulator in TMEM.  Both operands are K-major in the no-swizzle
// canonical layout.  The input window of 132 positions is stored as [chunk of
// 8 channels][position][8] (a bulk copy per chunk), so every 8 consecutive
// positions of a chunk are one core matrix and tap j is the same descriptor
// moved by j rows (16 bytes): A(j) = window rows j .. j + 127.  The weights w
// come in staging order (wstage_index: [K chunk = (j, 8 channels)][co][8]),
// one bulk copy per persistent CTA, which then walks the items with a grid
// stride as a pipeline: the copy warp
// fills kConvStages window stages ahead of the tensor cores, the tensor cores
// write two accumulators in turn, and the epilogue warps read one (position
// 32 (w % 4) + lane of the tile, channel group w / 4) while the next item's
// products go to the other.  The stages and accumulators hand over by
// mbarriers (copies -> full, products -> empty and tfull, accumulator read ->
// tempty).  A wait that gives up sets bit 1 of *err and ends the CTA's work.
template <int CIN, int COUT, int EPI>
__global__ void __launch_bounds__(role_threads(conv_epi_warps(COUT)), 2)
    conv_kernel(const bf16 *__restrict__ in, const bf16 *__restrict__ w, const float *__restrict__ bias,
                const int *__restrict__ periodic, int X, int B, void *__restrict__ out, const bf16 *__restrict__ mask,
                const float *__restrict__ edge, unsigned *__restrict__ err)
{
    static_assert(CIN % 16 == 0 && COUT % 16 == 0 && COUT <= 64, "padded channels");
    constexpr int EW = conv_epi_warps(COUT), CG = EW / 4;  // epilogue warps, channel groups
    constexpr int NCG = COUT / CG;                        // channels of a group
    constexpr int kCopy = EW, kMma = EW + 1;
    constexpr int KC = CIN / 8;                           // 8-channel chunks of a position
    constexpr int ROWS = kConvM + kTaps - 1;              // window positions
    constexpr int WCH = kTaps * KC;                       // weight chunks along K
    constexpr int NS = kConvStages;
    constexpr uint32_t ALBO = ROWS * 16, BLBO = COUT * 16;
    constexpr uint32_t ACOL = COUT < 32 ? 32 : COUT;      // TMEM columns of one accumulator (a power of 2)
    constexpr int kWin = KC * ROWS * 8;                   // bf16 per window stage
    extern __shared__ __align__(128) unsigned char smem[];
    bf16 *const ws = reinterpret_cast<bf16 *>(smem);      // [WCH][COUT][8]
    bf16 *const win_base = ws + WCH * COUT * 8;           // NS stages of [KC][ROWS][8]
    __shared__ __align__(8) uint64_t full[NS], empty[NS], tfull[2], tempty[2], done, wbar;
    __shared__ __align__(16) float s_bias[COUT];
    __shared__ uint32_t s_taddr;
    __shared__ int s_abort;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 32);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], 32 * EW);
        }
        mbar_init(&done, 1);
        mbar_init(&wbar, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        // the layer's weights, already in staging order (see wstage_index)
        constexpr uint32_t wbytes = uint32_t(WCH) * COUT * 16;
        mbar_arrive_tx(&wbar, wbytes);
        bulk_g2s(ws, w, wbytes, &wbar);
    }
    if (warp == kMma) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_taddr)),
                     "r"(2 * ACOL)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    pdl_wait();
    if (t == 0) pdl_trigger();
    const uint32_t taddr = s_taddr;
    const int tiles = (X + kConvM - 1) / kConvM, nitems = B * tiles;
    volatile int *const abort = &s_abort;
    if (warp == kCopy) {
        // the window of item `it` into stage it % NS once the products of item it - NS have read it
        int it = 0;
        for (int item = blockIdx.x; item < nitems; item += gridDim.x, ++it) {
            const int s = it % NS;
            if (it >= NS && !mbar_wait(&empty[s], (it / NS - 1) & 1, abort)) {
                give_up(abort, err);
                break;
            }
            const int b = item / tiles;
            const int mode = periodic[b] != 0 ? PAD_PERIODIC : (EPI == EPI_MASK_BF16 ? PAD_ZERO : PAD_REPLICATE);
            fill_rows<CIN>(win_base + s * kWin, in, b, (item % tiles) * kConvM, 2, ROWS, X, mode, lane, &full[s]);
        }
        drain_fills(full, NS, it);
        mbar_wait(&wbar, 0, nullptr);
    } else if (warp == kMma) {
        if (lane == 0) {
            int it = 0;
            for (int item = blockIdx.x; item < nitems; item += gridDim.x, ++it) {
                const int s = it % NS, a = it & 1;
                if ((it == 0 && !mbar_wait(&wbar, 0, abort)) || !mbar_wait(&full[s], (it / NS) & 1, abort) ||
                    (it >= 2 && !mbar_wait(&tempty[a], ((it >> 1) - 1) & 1, abort))) {
                    give_up(abort, err);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t wa = smem_u32(win_base + s * kWin), wb = smem_u32(ws);
                int step = 0;
#pragma unroll
                for (int j = 0; j < kTaps; ++j)
#pragma unroll
                    for (int kc = 0; kc < KC; kc += 2, ++step)
                        umma_bf16(taddr + a * ACOL, umma_desc(wa + kc * ALBO + j * 16, ALBO, 128),
                                  umma_desc(wb + (j * KC + kc) * BLBO, BLBO, 128), umma_idesc_bf16(kConvM, COUT),
                                  step);
                umma_commit(&empty[s]);
                umma_commit(&tfull[a]);
            }
            // every product has landed before the accumulators are freed
            umma_commit(&done);
            if (!mbar_wait(&done, 0, nullptr)) give_up(abort, err);
        }
        __syncwarp();
    } else {
        const int m = 32 * (warp & 3) + lane;  // position of the tile = TMEM lane
        const int c0 = (warp >> 2) * NCG;      // first channel of this thread's group
        if (EPI != EPI_MASK_BF16) {
            for (int e = t; e < COUT; e += 32 * EW) s_bias[e] = bias[e];
            asm volatile("bar.sync 1, %0;" ::"n"(32 * EW) : "memory");  // the epilogue warps only
        }
        int it = 0;
        for (int item = blockIdx.x; item < nitems; item += gridDim.x, ++it) {
            const int a = it & 1, b = item / tiles, x = (item % tiles) * kConvM + m;
            const bool valid = x < X;
            // the ReLU mask of the backward pass, loaded while the tensor cores work
            uint4 mk[EPI == EPI_MASK_BF16 ? NCG / 8 : 1];
            if constexpr (EPI == EPI_MASK_BF16) {
#pragma unroll
                for (int v = 0; v < NCG / 8; ++v)
                    mk[v] = valid ? *reinterpret_cast<const uint4 *>(mask + cm_index(b, x, c0 + 8 * v, COUT, X, 8))
                                  : make_uint4(0u, 0u, 0u, 0u);
            }
            // warp-uniform: tcgen05.ld below is issued by whole warps
            if (!__all_sync(0xffffffffu, mbar_wait(&tfull[a], (it >> 1) & 1, abort))) {
                give_up(abort, err);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            uint32_t r[NCG];
#pragma unroll
            for (int q = 0; q < NCG; q += 16)
                tmem_ld16(r + q, taddr + (uint32_t(32 * (warp & 3)) << 16) + a * ACOL + c0 + q);
            tmem_wait(r);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(&tempty[a]);  // the tensor cores may now overwrite this accumulator
            if (!valid) continue;
            float v[NCG];
#pragma unroll
            for (int q = 0; q < NCG; ++q) v[q] = __uint_as_float(r[q]);
            if constexpr (EPI != EPI_MASK_BF16) {
#pragma unroll
                for (int q = 0; q < NCG; q += 4) {
                    const float4 bb = *reinterpret_cast<const float4 *>(s_bias + c0 + q);
                    v[q] += bb.x;
                    v[q + 1] += bb.y;
                    v[q + 2] += bb.z;
                    v[q + 3] += bb.w;
                }
            }
            if constexpr (EPI == EPI_F32) {
                float *o = static_cast<float *>(out);
#pragma unroll
                for (int q = 0; q < NCG; q += 4)
                    *reinterpret_cast<float4 *>(o + cm_index(b, x, c0 + q, COUT, X, 4)) =
                        make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
                continue;
            }
            if constexpr (EPI == EPI_MASK_BF16) {
                if (periodic[b] == 0 && (x == 0 || x == X - 1)) {
                    const float *eg = edge + (size_t(b) * 2 + (x != 0)) * COUT + c0;
#pragma unroll
                    for (int q = 0; q < NCG; ++q) v[q] += eg[q];
                }
                const __nv_bfloat162 *mp = reinterpret_cast<const __nv_bfloat162 *>(mk);
#pragma unroll
                for (int q = 0; q < NCG / 2; ++q) {
                    const __nv_bfloat162 mv = mp[q];
                    v[2 * q] = __bfloat162float(mv.x) > 0.f ? v[2 * q] : 0.f;
                    v[2 * q + 1] = __bfloat162float(mv.y) > 0.f ? v[2 * q + 1] : 0.f;
                }
            } else {
#pragma unroll
                for (int q = 0; q < NCG; ++q) v[q] = fmaxf(v[q], 0.f);
            }
            bf16 *o = static_cast<bf16 *>(out);
#pragma unroll
            for (int q = 0; q < NCG; q += 8) {
                uint4 pk;
                __nv_bfloat162 *pp = reinterpret_cast<__nv_bfloat162 *>(&pk);
#pragma unroll
                for (int h = 0; h < 4; ++h) pp[h] = __floats2bfloat162_rn(v[q + 2 * h], v[q + 2 * h + 1]);
                *reinterpret_cast<uint4 *>(o + cm_index(b, x, c0 + q, COUT, X, 8)) = pk;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == kMma) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(2 * ACOL) : "memory");
    }
}

// Weight and bias gradients of one layer on the tensor cores:
//   dW[co][j][ci] = sum_{b,x} dz[b][x][co] in[b][x + j - 2][ci],  db[co] = sum dz[b][x][co].
// Per tap j a GEMM over K = positions, accumulated in TMEM over every (sample,
// 128-position tile) item of the CTA: the operand with 64 channels is A (M =
// 64), the other B (N = its channel count), D_j in TMEM columns [j N, (j + 1) N).
// Both operands are MN-major in the no-swizzle canonical layout, staged as
// [chunk of 8 channels][position][8] (a bulk copy per chunk of the
// chunk-major tensors): 8 consecutive positions of a chunk are one core
// matrix, the next 8 positions follow at 128 bytes (LBO) and the next chunk at
// a whole chunk's rows (SBO); tap j of the input window is the same descriptor
// moved by j rows.  An M = 64 accumulator keeps row m in TMEM lane
// 32 (m / 16) + m % 16.  The copy warp fills kWgradStages stages ahead of the
// tensor cores; a stage is free again once its products have completed and
// the epilogue warps have added its dz tile into their bias-gradient partial
// sums (empty: one commit + 128 arrivals).  Each CTA writes one partial
// [co][5 cin] + [co]; reduce_partials_kernel sums the partials in a fixed
// order.  A wait that gives up sets bit 1 of *err and ends the CTA's work.
template <int CIN, int COUT>
__global__ void __launch_bounds__(role_threads(kWgradEpiWarps), 1)
    wgrad_kernel(const bf16 *__restrict__ dz, const bf16 *__restrict__ in, const int *__restrict__ periodic, int X,
                 int ntiles, float *__restrict__ partial, unsigned *__restrict__ err)
{
    static_assert((COUT == 64 && (CIN == 16 || CIN == 64)) || (COUT == 16 && CIN == 64), "layer shapes");
    constexpr bool DZ_A = COUT == 64;           // A = dz (M = cout); else A = input window (M = cin)
    constexpr int NB = DZ_A ? CIN : COUT;       // N of one tap
    constexpr int KCD = COUT / 8, KCI = CIN / 8;
    constexpr int RD = kConvM, RI = kConvM + kTaps - 1;  // staged positions of dz and of the input window
    constexpr uint32_t SD = RD * 16, SI = RI * 16;       // chunk strides (bytes)
    constexpr int NTOT = kTaps * NB, NS = kWgradStages;
    constexpr int kCopy = kWgradEpiWarps, kMma = kWgradEpiWarps + 1;
    constexpr uint32_t NCOL = NTOT <= 32 ? 32 : (NTOT <= 64 ? 64 : (NTOT <= 128 ? 128 : (NTOT <= 256 ? 256 : 512)));
    constexpr int kStage = KCD * RD * 8 + KCI * RI * 8;  // bf16 per stage
    // bias gradient: epilogue warp w sums dz chunks w and w + 4 (those below KCD),
    // lane l the rows l, l + 32, l + 64, l + 96 of each tile
    constexpr int DBC = KCD > 4 ? 2 : 1;
    extern __shared__ __align__(128) unsigned char smem[];
    bf16 *const stage_base = reinterpret_cast<bf16 *>(smem);
    __shared__ __align__(8) uint64_t full[NS], empty[NS], done;
    __shared__ uint32_t s_taddr;
    __shared__ int s_abort;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int tiles = (X + kConvM - 1) / kConvM;
    if (t == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 64);
            mbar_init(&empty[s], 1 + 32 * kWgradEpiWarps);
        }
        mbar_init(&done, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMma) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_taddr)),
                     "r"(NCOL)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    pdl_wait();
    if (t == 0) pdl_trigger();
    const uint32_t taddr = s_taddr;
    volatile int *const abort = &s_abort;
    int nit = 0;  // items of this CTA
    for (int item = blockIdx.x; item < ntiles; item += gridDim.x) ++nit;
    if (warp == kCopy) {
        // dz rows x0 .. x0 + 127 (zero beyond the sample), input window rows x0 - 2 ..
        // x0 + 129 (periodic or replicated ends): two fills, 64 arrivals on full
        int it = 0;
        for (int item = blockIdx.x; item < ntiles; item += gridDim.x, ++it) {
            const int s = it % NS;
            if (it >= NS && !mbar_wait(&empty[s], (it / NS - 1) & 1, abort)) {
                give_up(abort, err);
                break;
            }
            const int b = item / tiles, x0 = (item % tiles) * kConvM;
            bf16 *sdz = stage_base + s * kStage;
            fill_rows<COUT>(sdz, dz, b, x0, 0, RD, X, PAD_ZERO, lane, &full[s]);
            fill_rows<CIN>(sdz + KCD * RD * 8, in, b, x0, 2, RI, X, periodic[b] != 0 ? PAD_PERIODIC : PAD_REPLICATE,
                           lane, &full[s]);
        }
        drain_fills(full, NS, it);
    } else if (warp == kMma) {
        if (lane == 0) {
            constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                                       (uint32_t(NB >> 3) << 17) | (uint32_t(64 >> 4) << 24);  // MN-major A and B, M = 64
            for (int it = 0; it < nit; ++it) {
                const int s = it % NS;
                if (!mbar_wait(&full[s], (it / NS) & 1, abort)) {
                    give_up(abort, err);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t ad = smem_u32(stage_base + s * kStage), ai = ad + KCD * RD * 16;
#pragma unroll
                for (int j = 0; j < kTaps; ++j)
#pragma unroll
                    for (int k0 = 0; k0 < kConvM; k0 += 16) {
                        const uint64_t dd = umma_desc(ad + k0 * 16, 128, SD);
                        const uint64_t di = umma_desc(ai + (k0 + j) * 16, 128, SI);
                        umma_bf16(taddr + j * NB, DZ_A ? dd : di, DZ_A ? di : dd, idesc, it > 0 || k0 > 0);
                    }
                umma_commit(&empty[s]);
            }
            umma_commit(&done);
            if (!mbar_wait(&done, 0, nullptr)) give_up(abort, err);
        }
        __syncwarp();
    } else {
        float db[DBC][8];
#pragma unroll
        for (int d = 0; d < DBC; ++d)
#pragma unroll
            for (int k = 0; k < 8; ++k) db[d][k] = 0.f;
        bool ok = true;
        for (int it = 0; it < nit; ++it) {
            const int s = it % NS;
            if (!mbar_wait(&full[s], (it / NS) & 1, abort)) {
                give_up(abort, err);
                ok = false;
                break;
            }
            const bf16 *sdz = stage_base + s * kStage;
#pragma unroll
            for (int d = 0; d < DBC; ++d) {
                const int c = warp + 4 * d;
                if (c < KCD)
#pragma unroll
                    for (int r = 0; r < RD; r += 32) {
                        const uint4 u = *reinterpret_cast<const uint4 *>(sdz + (c * RD + r + lane) * 8);
                        const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            db[d][2 * k] += __bfloat162float(h[k].x);
                            db[d][2 * k + 1] += __bfloat162float(h[k].y);
                        }
                    }
            }
            mbar_arrive(&empty[s]);
        }
        // every epilogue warp has read its last dz tile before the stage buffers
        // are reused below (also one that gave up)
        asm volatile("bar.sync 1, %0;" ::"n"(32 * kWgradEpiWarps) : "memory");
        // the lane sums of each column, in a fixed order
#pragma unroll
        for (int d = 0; d < DBC; ++d)
#pragma unroll
            for (int k = 0; k < 8; ++k)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) db[d][k] += __shfl_xor_sync(0xffffffffu, db[d][k], o);
        // the accumulators once every product of the CTA has landed
        if (!__all_sync(0xffffffffu, ok && mbar_wait(&done, 0, abort))) {  // warp-uniform, as tcgen05.ld
            if (ok) give_up(abort, err);
            ok = false;
        }
        if (ok) {
            // the accumulators go through shared memory (the idle stage buffers) as
            // [co][5 cin] rows padded by one word, then out in coalesced rows
            constexpr int RW = kTaps * CIN, RP = RW + 1;
            static_assert(COUT * RP * 4 <= NS * kStage * 2, "transpose buffer");
            float *T = reinterpret_cast<float *>(smem);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // after the tensor cores' reads
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // lane l < 16 of warp w holds row m = 16 w + l of every D_j; 64 columns per wait
            const int m = 16 * warp + lane;
            static_assert(NTOT % 16 == 0, "whole 16-column loads");
#pragma unroll 1
            for (int c0 = 0; c0 < NTOT; c0 += 64) {
                uint32_t r[64];
#pragma unroll
                for (int h = 0; h < 4; ++h)
                    if (c0 + 16 * h < NTOT) tmem_ld16(r + 16 * h, taddr + (uint32_t(warp * 32) << 16) + c0 + 16 * h);
                tmem_wait(r);
                if (lane < 16) {
#pragma unroll
                    for (int q = 0; q < 64; ++q) {
                        const int col = c0 + q, j = col / NB, n = col % NB;  // tap j, channel n of B
                        // DZ_A: m = co, n = ci; else m = ci, n = co
                        const int co = DZ_A ? m : n, ci = DZ_A ? n : m;
                        if (col < NTOT) T[co * RP + j * CIN + ci] = nit > 0 ? __uint_as_float(r[q]) : 0.f;
                    }
                }
            }
        }
        // every epilogue warp, also one that gave up (the transpose buffer is shared)
        asm volatile("bar.sync 1, %0;" ::"n"(32 * kWgradEpiWarps) : "memory");
        if (ok) {
            constexpr int RW = kTaps * CIN, RP = RW + 1;
            const float *T = reinterpret_cast<const float *>(smem);
            float *P = partial + size_t(blockIdx.x) * (COUT * RW + COUT);
            static_assert(RW % 4 == 0, "rows of whole float4");
            for (int e = 4 * t; e < COUT * RW; e += 4 * 32 * kWgradEpiWarps) {
                const float *src = T + (e / RW) * RP + e % RW;  // four values of one row
                *reinterpret_cast<float4 *>(P + e) = make_float4(src[0], src[1], src[2], src[3]);
            }
            if (lane == 0)
#pragma unroll
                for (int d = 0; d < DBC; ++d) {
                    const int c = warp + 4 * d;
                    if (c < KCD)
#pragma unroll
                        for (int k = 0; k < 8; ++k) P[size_t(COUT) * RW + 8 * c + k] = db[d][k];
                }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == kMma) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(NCOL) : "memory");
    }
}

// Replicate padding feeds the end values a[0] and a[X-1] of a sample into the
// taps that reach past its ends, so their gradients get terms the zero-padded
// transposed convolution lacks:
//   left  (x = 0):     sum_co (W0 + W1)[co][ci] dz[0][co] + W0[co][ci] dz[1][co]
//   right (x = X - 1): sum_co (W3 + W4)[co][ci] dz[X-1][co] + W4[co][ci] dz[X-2][co]
// w is the forward layer's W[co][j][ci] (staging order); dz is chunk-major.  One block per side, kEdgeSamples
// samples and kEdgeChannels input channels: the two weight combinations of
// that side and channel range (the same for every sample) and the samples' end
// gradients are staged in shared memory once.
constexpr int kEdgeSamples = 16, kEdgeChannels = 16;
__global__ void __launch_bounds__(256) edge_grad_kernel(const bf16 *__restrict__ dz, const bf16 *__restrict__ w,
                                                        const int *__restrict__ periodic, int B, int X, int cout,
                                                        int cin, float *__restrict__ edge)
{
    pdl_wait();
    pdl_trigger();
    __shared__ float s_a[64][kEdgeChannels], s_n[64][kEdgeChannels];  // [co][ci - c0], cout <= 64
    __shared__ float s_d0[kEdgeSamples][64], s_d1[kEdgeSamples][64];
    const int side = blockIdx.y, b0 = blockIdx.x * kEdgeSamples, c0 = blockIdx.z * kEdgeChannels, t = threadIdx.x;
    const int ja = side ? 3 : 0, jb = side ? 4 : 1, jn = side ? 4 : 0;
    for (int e = t; e < cout * kEdgeChannels; e += blockDim.x) {
        const int co = e / kEdgeChannels, cc = e - co * kEdgeChannels, ci = c0 + cc;
        float a = 0.f, n = 0.f;
        if (ci < cin) {
            a = __bfloat162float(w[wstage_index(co, ja, ci, cout, cin)]) +
                __bfloat162float(w[wstage_index(co, jb, ci, cout, cin)]);
            n = __bfloat162float(w[wstage_index(co, jn, ci, cout, cin)]);
        }
        s_a[co][cc] = a;
        s_n[co][cc] = n;
    }
    for (int e = t; e < kEdgeSamples * cout; e += blockDim.x) {
        const int sm = e / cout, co = e - sm * cout, b = b0 + sm;
        float d0 = 0.f, d1 = 0.f;
        if (b < B) {
            d0 = __bfloat162float(dz[cm_index(b, side ? X - 1 : 0, co, cout, X, 8)]);
            d1 = __bfloat162float(dz[cm_index(b, side ? X - 2 : 1, co, cout, X, 8)]);
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
    pdl_wait();
    pdl_trigger();
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

// Network inputs are padded to this many channels (two 16-byte rows).
constexpr int kInPad = 16;

// Position pos = b X + p of the input: sample k's features (f32 [n][X][cin],
// cin <= kInPad) normalised, stored bf16 chunk-major with kInPad channels.
__device__ __forceinline__ void pack_position(const float *__restrict__ x, int64_t k, int64_t b, int p, int X,
                                              int cin, const float *__restrict__ shift,
                                              const float *__restrict__ inv_scale, bf16 *__restrict__ out)
{
    float v[kInPad];
#pragma unroll
    for (int c = 0; c < kInPad; ++c) v[c] = c < cin ? (x[(k * X + p) * cin + c] - shift[c]) * inv_scale[c] : 0.f;
#pragma unroll
    for (int q = 0; q < kInPad / 8; ++q) {
        uint4 pk;
        __nv_bfloat162 *pp = reinterpret_cast<__nv_bfloat162 *>(&pk);
#pragma unroll
        for (int h = 0; h < 4; ++h) pp[h] = __floats2bfloat162_rn(v[8 * q + 2 * h], v[8 * q + 2 * h + 1]);
        *reinterpret_cast<uint4 *>(out + cm_index(b, p, 8 * q, kInPad, X, 8)) = pk;
    }
}

// Input features (f32 [B][X][cin]) -> the network's input; one thread per position.
__global__ void pack_input_kernel(const float *__restrict__ x, int64_t npos, int X, int cin,
                                  const float *__restrict__ shift, const float *__restrict__ inv_scale,
                                  bf16 *__restrict__ out)
{
    pdl_wait();
    pdl_trigger();
    const int64_t pos = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (pos >= npos) return;
    pack_position(x, pos / X, pos / X, int(pos % X), X, cin, shift, inv_scale, out);
}

// The same for the mini-batch idx[0..B) = perm[step B ..] (step read from the
// device) of a data set of n samples (X positions each), with the samples'
// padding kinds gathered into perb.  An index outside
// [0, n) sets *bad and reads sample 0 instead, so nothing is read out of bounds.
__global__ void pack_gather_kernel(const float *__restrict__ x, const int32_t *__restrict__ per,
                                   const int32_t *__restrict__ perm, const int *__restrict__ step, int64_t n, int B,
                                   int X, int cin, const float *__restrict__ shift,
                                   const float *__restrict__ inv_scale, bf16 *__restrict__ out,
                                   int32_t *__restrict__ perb, unsigned *__restrict__ bad)
{
    pdl_wait();
    pdl_trigger();
    const int32_t *__restrict__ idx = perm + int64_t(*step) * B;  // this step's samples
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e < B) {
        const int64_t k = idx[e];
        const bool ok = k >= 0 && k < n;
        if (!ok) atomicOr(bad, 1u);
        perb[e] = per[ok ? k : 0];
    }
    if (e >= int64_t(B) * X) return;
    const int64_t b = e / X;
    int64_t k = idx[b];
    if (k < 0 || k >= n) k = 0;
    pack_position(x, k, b, int(e % X), X, cin, shift, inv_scale, out);
}

// Output channels of the last layer as computed: four 16-byte rows of 4 f32 in
// the prediction, two rows of 8 bf16 in its gradient.
constexpr int kOutPad = 16;
// Blocks (and loss partials) of mse_kernel for npos positions.
inline unsigned mse_blocks(int64_t npos) { return unsigned((npos + 255) / 256); }

// Mean squared error between prediction (f32 chunk-major in rows of 4, kOutPad
// channels, first cout used) and target / out_scale; writes dL/dpred (bf16
// chunk-major, padded channels zero) and per-block partial sums of the squared
// error (256 threads, one per position).
// y rows of the batch: y[b] directly, or y[idx[b]] of the whole data set
// (idx already checked by pack_gather_kernel; X positions per sample).
__global__ void __launch_bounds__(256) mse_kernel(const float *__restrict__ pred, const float *__restrict__ y,
                                                  const int32_t *__restrict__ idx, const int *__restrict__ step, int X,
                                                  int64_t npos, int cout, const float *__restrict__ inv_out_scale,
                                                  float grad_scale, bf16 *__restrict__ dpred,
                                                  float *__restrict__ partial)
{
    pdl_wait();
    pdl_trigger();
    // step (device, may be null): the batch is idx[step * B ..] of a training run's permutation
    if (idx && step) idx += int64_t(*step) * (npos / X);
    __shared__ float red[8];
    const int64_t pos = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    float se = 0.f;
    if (pos < npos) {
        const int64_t b = pos / X;
        const int p = int(pos % X);
        const int64_t row = (idx ? int64_t(idx[b]) : b) * X + p;
        float g[kOutPad];
#pragma unroll
        for (int q = 0; q < kOutPad / 4; ++q) {
            const float4 pr = *reinterpret_cast<const float4 *>(pred + cm_index(b, p, 4 * q, kOutPad, X, 4));
            const float pv[4] = {pr.x, pr.y, pr.z, pr.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int c = 4 * q + k;
                float d = 0.f;
                if (c < cout) {
                    d = pv[k] - y[row * cout + c] * inv_out_scale[c];
                    se += d * d;
                }
                g[c] = grad_scale * d;
            }
        }
#pragma unroll
        for (int q = 0; q < kOutPad / 8; ++q) {
            uint4 pk;
            __nv_bfloat162 *pp = reinterpret_cast<__nv_bfloat162 *>(&pk);
#pragma unroll
            for (int h = 0; h < 4; ++h) pp[h] = __floats2bfloat162_rn(g[8 * q + 2 * h], g[8 * q + 2 * h + 1]);
            *reinterpret_cast<uint4 *>(dpred + cm_index(b, p, 8 * q, kOutPad, X, 8)) = pk;
        }
    }
    // block sum in a fixed order: lanes by shuffles, then the 8 warps in turn
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = se;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < 8; ++w) t += red[w];
        partial[blockIdx.x] = t;
    }
}

// Prediction in physical units: y[b][x][c] = pred(b, x, c) * out_scale[c], c < cout
// (pred chunk-major f32 in rows of 4, coutp channels).
__global__ void unpack_output_kernel(const float *__restrict__ pred, int64_t npos, int X, int cout, int coutp,
                                     const float *__restrict__ out_scale, float *__restrict__ y)
{
    pdl_wait();
    pdl_trigger();
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= npos * cout) return;
    const int64_t pos = e / cout;
    const int c = int(e % cout);
    y[e] = pred[cm_index(pos / X, pos % X, c, coutp, X, 4)] * out_scale[c];
}

// Mean loss of one batch from the per-block partial sums of mse_kernel, summed
// in a fixed order by one block of 256 threads: each thread adds its strided
// share in FP32, the thread sums are combined in FP64.
__global__ void loss_sum_kernel(const float *__restrict__ partial, int nparts, float scale, float *__restrict__ out,
                                const int *__restrict__ step)
{
    pdl_wait();
    pdl_trigger();
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
__global__ void step_inc_kernel(int *step)
{
    pdl_wait();
    pdl_trigger();
    *step += 1;
}

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
    // transposed, into wt16 at the same offset (both in staging order)
    bf16 *w16, *wt16;
    int nl;
    int64_t woff[kAdamLayers];
    int cout[kAdamLayers], cin[kAdamLayers];
};
__global__ void adam_kernel(AdamArgs a)
{
    pdl_wait();
    pdl_trigger();
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
            a.w16[a.woff[l] + wstage_index(co, j, ci, cout_, ci_)] = b;
            a.wt16[a.woff[l] + wstage_index(ci, kTaps - 1 - j, co, ci_, cout_)] = b;
            break;
        }
    }
}

// bf16 copies of one layer's weights, in staging order (wstage_index): w =
// W[co][j][ci] and wt = the transposed convolution's W[ci][4 - j][co].
__global__ void cast_weights_kernel(const float *__restrict__ wf, int cout, int cin, bf16 *__restrict__ w,
                                    bf16 *__restrict__ wt)
{
    pdl_wait();
    pdl_trigger();
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= cout * kTaps * cin) return;
    const int co = e / (kTaps * cin), j = (e / cin) % kTaps, ci = e % cin;
    const bf16 v = __float2bfloat16(wf[e]);
    w[wstage_index(co, j, ci, cout, cin)] = v;
    wt[wstage_index(ci, kTaps - 1 - j, co, cin, cout)] = v;
}

// ---------------------------------------------------------------------------
struct Layer {
    int cin, cout;    // padded
    int cin_real, cout_real;
    int64_t woff, boff;  // offsets of W [cout][5][cin] and bias [cout] in the f32 parameter vector
};

// Launches kernel k on stream s with programmatic stream serialisation (see
// pdl_wait): it may start before the previous kernel in the stream ends.
template <typename... KArgs, typename... Args>
cudaError_t launch(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

// CTAs per SM of a tensor-core kernel: as many as shared memory and the 512
// TMEM columns of an SM hold (each CTA allocates tmem_cols for the whole
// launch), at most cap.  Sets the kernel's shared-memory limit on the current
// device the first time, and remembers the result per device in the kernel's
// own cache ({CTAs per SM, SMs} + 1; 0: not known yet).
typedef std::atomic<int> ShapeCache[kMaxDevices][2];
template <typename K>
cudaError_t ctas_per_sm(K k, int threads, size_t smem, int tmem_cols, int cap, ShapeCache &cache, int *per_sm,
                        int *sms)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < kMaxDevices && cache[dev][0].load() > 0) {
        *per_sm = cache[dev][0].load() - 1;
        *sms = cache[dev][1].load() - 1;
        return cudaSuccess;
    }
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    // all of the SM's unified L1 / shared memory as shared memory, so that the
    // occupancy below counts every CTA the SM's shared memory can hold
    e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, int(cudaSharedmemCarveoutMaxShared));
    if (e != cudaSuccess) return e;
    int occ = 0, n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, threads, smem);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    // the same bound from the SM's shared memory, registers (allocated per warp
    // in units of 256) and threads; the larger of the two counts is used (a grid
    // above what fits only queues CTAs, it stays correct)
    cudaFuncAttributes fa;
    int smem_sm = 0, resv = 0, regs_sm = 0, thr_sm = 0;
    if (cudaFuncGetAttributes(&fa, k) == cudaSuccess &&
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) == cudaSuccess) {
        const int by_smem = smem_sm / int(smem + fa.sharedSizeBytes + size_t(resv));
        const int warp_regs = (fa.numRegs * 32 + 255) / 256 * 256;
        const int by_regs = regs_sm / std::max(1, warp_regs * (threads / 32));
        occ = std::max(occ, std::min(std::min(by_smem, by_regs), thr_sm / threads));
    }
    *per_sm = std::max(1, std::min(std::min(occ, 512 / tmem_cols), cap));
    *sms = std::max(1, n);
    if (dev >= 0 && dev < kMaxDevices) {
        cache[dev][1].store(*sms + 1);
        cache[dev][0].store(*per_sm + 1);
    }
    return cudaSuccess;
}

// Persistent grid of the convolution: every CTA an SM holds, at most one per item.
template <int CIN, int COUT, int EPI>
cudaError_t conv_launch(const bf16 *in, const bf16 *w, const float *bias, const int *per, int B, int X, void *out,
                        const bf16 *mask, const float *edge, unsigned *err, cudaStream_t s)
{
    constexpr size_t smem =
        16 * (size_t(kTaps) * (CIN / 8) * COUT + size_t(kConvStages) * (CIN / 8) * (kConvM + kTaps - 1));
    constexpr int ncol = 2 * (COUT < 32 ? 32 : COUT);
    auto k = conv_kernel<CIN, COUT, EPI>;
    constexpr int threads = role_threads(conv_epi_warps(COUT));
    static ShapeCache cache;
    int per_sm = 0, sms = 0;
    cudaError_t e = ctas_per_sm(k, threads, smem, ncol, 8, cache, &per_sm, &sms);
    if (e != cudaSuccess) return e;
    const int items = B * ((X + kConvM - 1) / kConvM);
    const int grid = std::max(1, std::min(items, sms * per_sm));
    return launch(k, dim3(grid), dim3(threads), smem, s, in, w, bias, per, X, B, out, mask, edge, err);
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

// The weight-gradient grid: CTAs per SM by shared memory and by the TMEM
// columns of their five accumulators, at most 2 (the partial buffer holds
// 2 x SMs parts); *parts receives the grid, the number of partials to sum.
template <int CIN, int COUT>
cudaError_t wgrad_launch(const bf16 *dz, const bf16 *in, const int *per, int B, int X, int sms, float *partial,
                         unsigned *err, int *parts, cudaStream_t s)
{
    constexpr int RD = kConvM, RI = kConvM + kTaps - 1;
    constexpr size_t smem = size_t(kWgradStages) * 16 * (size_t(COUT / 8) * RD + size_t(CIN / 8) * RI);
    constexpr int ntot = kTaps * (COUT == 64 ? CIN : COUT);
    constexpr int ncol = ntot <= 32 ? 32 : (ntot <= 64 ? 64 : (ntot <= 128 ? 128 : (ntot <= 256 ? 256 : 512)));
    auto k = wgrad_kernel<CIN, COUT>;
    constexpr int threads = role_threads(kWgradEpiWarps);
    static ShapeCache cache;
    int per_sm = 0, dev_sms = 0;
    cudaError_t e = ctas_per_sm(k, threads, smem, ncol, 2, cache, &per_sm, &dev_sms);
    if (e != cudaSuccess) return e;
    const int ntiles = B * ((X + kConvM - 1) / kConvM);
    const int grid = std::max(1, std::min(ntiles, std::max(1, sms) * per_sm));
    *parts = grid;
    return launch(k, dim3(grid), dim3(threads), smem, s, dz, in, per, X, ntiles, partial, err);
}

cudaError_t wgrad_any(int cin, int cout, const bf16 *dz, const bf16 *in, const int *per, int B, int X, int sms,
                      float *partial, unsigned *err, int *parts, cudaStream_t s)
{
    if (cin == 16 && cout == 64) return wgrad_launch<16, 64>(dz, in, per, B, X, sms, partial, err, parts, s);
    if (cin == 64 && cout == 64) return wgrad_launch<64, 64>(dz, in, per, B, X, sms, partial, err, parts, s);
    if (cin == 64 && cout == 16) return wgrad_launch<64, 16>(dz, in, per, B, X, sms, partial, err, parts, s);
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
    float *partial = nullptr;  // two halves of 2 x sms weight-gradient partials each
    // a second stream for the end terms and partial sums of the backward pass, and its events
    cudaStream_t side = nullptr;
    std::vector<cudaEvent_t> events;
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
    int sms = 0;  // SMs of the device; the weight-gradient partial buffer holds 2 x sms parts
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
    for (cudaEvent_t e : c->events) cudaEventDestroy(e);
    if (c->side) cudaStreamDestroy(c->side);
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
        QC_CUDA(c, launch(cast_weights_kernel, dim3((n + 255) / 256), dim3(256), 0, c->stream, c->param + L.woff,
                          L.cout, L.cin, c->w16 + L.woff, c->wt16 + L.woff));
    }
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
    QC_CUDA(c, launch(pack_input_kernel, dim3(unsigned((npos + 255) / 256)), dim3(256), 0, c->stream, x, npos,
                      c->d.positions, c->d.in_channels, c->norm, c->norm + 8, c->act[0]));
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
                          float *loss, float *losses = nullptr)
{
    const int X = c->d.positions, nl = int(c->layers.size());
    const int64_t npos = int64_t(B) * X;
    const unsigned nb = mse_blocks(npos);
    const float gscale = 2.f / float(npos * c->d.out_channels);
    QC_CUDA(c, launch(mse_kernel, dim3(nb), dim3(256), 0, c->stream, c->pred, y, yidx, ystep, X, npos,
                      c->d.out_channels, c->norm + 24, gscale, c->dz[nl - 1], c->loss_partial));
    // The weight gradients and backward-data convolutions run on c->stream; the end terms of
    // layer l (after dz[l] is written) and the sum of layer l's weight-gradient partials (after
    // they are written) run on a second stream beside them, joined by events: the end terms
    // before the backward-data convolution that adds them, every partial sum before the end of
    // the pass.  Layer l's partials sit in half l % 2 of the partial buffer, so that the next
    // layer's weight gradient does not wait for this layer's sum.
    // per layer l: [4 l] dz[l] ready, [4 l + 1] end terms, [4 l + 2] partials; [3] the join at the
    // end, [4 (nl - 1) + 3] the loss partials
    cudaEvent_t *ev = c->events.data();
    const size_t half = size_t(2 * c->sms) * (64 * kTaps * 64 + 64);
    if (losses) {
        // a training run's per-step loss (device array, slot *ystep), on the second stream
        QC_CUDA(c, cudaEventRecord(ev[4 * (nl - 1) + 3], c->stream));
        QC_CUDA(c, cudaStreamWaitEvent(c->side, ev[4 * (nl - 1) + 3], 0));
        QC_CUDA(c, launch(loss_sum_kernel, dim3(1), dim3(256), 0, c->side, c->loss_partial, int(nb),
                          float(1.0 / double(npos * c->d.out_channels)), losses, ystep));
    }
    for (int l = nl - 1; l >= 0; --l) {
        const Layer &L = c->layers[l];
        const int len = L.cout * kTaps * L.cin + L.cout;  // a multiple of 4 (channels are padded to 16)
        if (len % 4 != 0) return cfail(c, QL_EUNSUPPORTED, "channel padding");
        float *part = c->partial + (l % 2) * half;
        if (l > 0) {
            // end terms of replicate padding for dz[l-1], beside the weight gradient
            static_assert(kEdgeSamples * kEdgeChannels == 256, "one output per thread");
            QC_CUDA(c, cudaEventRecord(ev[4 * l], c->stream));
            QC_CUDA(c, cudaStreamWaitEvent(c->side, ev[4 * l], 0));
            QC_CUDA(c, launch(edge_grad_kernel,
                              dim3((B + kEdgeSamples - 1) / kEdgeSamples, 2, (L.cin + kEdgeChannels - 1) / kEdgeChannels),
                              dim3(256), 0, c->side, c->dz[l], c->w16 + L.woff, per, B, X, L.cout, L.cin, c->edge));
            QC_CUDA(c, cudaEventRecord(ev[4 * l + 1], c->side));
        }
        int parts = 0;
        QC_CUDA(c, wgrad_any(L.cin, L.cout, c->dz[l], c->act[l], per, B, X, c->sms, part, c->bad, &parts,
                             c->stream));
        // partial layout per CTA: [cout][5 cin] then [cout]; W and b are contiguous in the parameter vector
        QC_CUDA(c, cudaEventRecord(ev[4 * l + 2], c->stream));
        QC_CUDA(c, cudaStreamWaitEvent(c->side, ev[4 * l + 2], 0));
        QC_CUDA(c, launch(reduce_partials_kernel, dim3((len + 127) / 128), dim3(32 * kReduceWarps), 0, c->side,
                          part, parts, len, c->grad + L.woff));
        if (l > 0) {
            // dz[l-1] = (W^T * dz[l] + end terms of replicate padding) masked by act[l] > 0
            // (act[l] is the output of layer l-1)
            QC_CUDA(c, cudaStreamWaitEvent(c->stream, ev[4 * l + 1], 0));
            QC_CUDA(c, conv_any(L.cout, L.cin, EPI_MASK_BF16, c->dz[l], c->wt16 + L.woff, nullptr, per, B, X,
                                c->dz[l - 1], c->act[l], c->edge, c->bad, c->stream));
        }
    }
    // the side stream's last partial sum before anything that follows on c->stream
    QC_CUDA(c, cudaEventRecord(ev[3], c->side));
    QC_CUDA(c, cudaStreamWaitEvent(c->stream, ev[3], 0));
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
        L.cin = l == 0 ? kInPad : 64;
        L.cout = l == d->layers - 1 ? kOutPad : 64;
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
    c->pred = static_cast<float *>(calloc_dev(c, sizeof(float) * npos * kOutPad));
    c->norm = static_cast<float *>(calloc_dev(c, sizeof(float) * 32));
    for (int l = 0; l < d->layers; ++l) {
        c->act.push_back(static_cast<bf16 *>(calloc_dev(c, sizeof(bf16) * npos * c->layers[l].cin)));
        c->dz.push_back(static_cast<bf16 *>(calloc_dev(c, sizeof(bf16) * npos * c->layers[l].cout)));
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    c->sms = sms > 0 ? sms : 128;
    c->partial = static_cast<float *>(calloc_dev(c, sizeof(float) * 2 * size_t(2 * c->sms) * (64 * kTaps * 64 + 64)));
    if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess) c->side = nullptr;
    c->events.assign(size_t(4 * d->layers), nullptr);
    for (cudaEvent_t &e : c->events)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) e = nullptr;
    c->loss_partial = static_cast<float *>(calloc_dev(c, sizeof(float) * mse_blocks(npos)));
    c->edge = static_cast<float *>(calloc_dev(c, sizeof(float) * size_t(B) * 2 * 64));
    c->perb = static_cast<int32_t *>(calloc_dev(c, sizeof(int32_t) * size_t(B)));
    c->bad = static_cast<unsigned *>(calloc_dev(c, sizeof(unsigned)));
    bool ok = c->param && c->grad && c->m && c->v && c->w16 && c->wt16 && c->pred && c->norm && c->partial &&
              c->loss_partial && c->edge && c->perb && c->bad;
    for (int l = 0; l < d->layers; ++l) ok = ok && c->act[l] && c->dz[l];
    if (!ok) return bail(QL_ENOMEM, "closure allocation failed");
    bool evok = c->side != nullptr;
    for (cudaEvent_t e : c->events) evok = evok && e != nullptr;
    if (!evok) return bail(QL_ECUDA, "closure stream or event creation failed");

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
    QC_CUDA(c, launch(unpack_output_kernel, dim3(unsigned((npos * c->d.out_channels + 255) / 256)), dim3(256), 0,
                      c->stream, c->pred, npos, c->d.positions, c->d.out_channels, c->layers.back().cout, c->norm + 16,
                      y));
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
    QC_CUDA(c, launch(adam_kernel, dim3(unsigned((c->nparam + 255) / 256)), dim3(256), 0, c->stream, a));
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
    QC_CUDA(c, launch(pack_gather_kernel, dim3(unsigned((B * X + 255) / 256)), dim3(256), 0, c->stream, x, periodic,
                      perm, c->d_step, n, int(B), X, c->d.in_channels, c->norm, c->norm + 8, c->act[0], c->perb,
                      c->bad));
    ql_status st = forward(c, c->perb, int(B));
    if (st == QL_OK) st = backward(c, y, perm, c->d_step, c->perb, int(B), nullptr, losses);
    if (st != QL_OK) return st;
    AdamArgs a = adam_args(c);
    a.step = c->d_step;
    a.lr_arr = c->d_sched;
    a.c1_arr = c->d_sched + c->sched_cap;
    a.c2_arr = c->d_sched + 2 * c->sched_cap;
    QC_CUDA(c, launch(adam_kernel, dim3(unsigned((c->nparam + 255) / 256)), dim3(256), 0, c->stream, a));
    if (!a.nl) {
        st = refresh_weights(c);
        if (st != QL_OK) return st;
    }
    QC_CUDA(c, launch(step_inc_kernel, dim3(1), dim3(1), 0, c->stream, c->d_step));
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
