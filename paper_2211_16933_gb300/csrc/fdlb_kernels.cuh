// Device code of the finite-difference Enskog-Shakhov lattice Boltzmann
// solver, templated on the arithmetic type (float or double) and the
// velocity-set size Q.  Included by fdlb_f32.cu and fdlb_f64.cu, which
// define QL_TAB (the per-precision __constant__ table) before including it.
//
// One launch of fdlb_stage_kernel performs one stage of the third-order TVD
// Runge-Kutta scheme (App. A.1, Eq. rk3) for every (cell, velocity) pair:
//   moments (Sec. II.D) -> eta, chi, b rho chi, tau, Pr (Secs. II.A-B)
//   -> 6th-order gradients of ln rho, u, ln T (App. A.3)
//   -> discrete equilibrium n g_k (Eq. feq) -> Shakhov targets (Sec. II.C)
//   -> J1 (Eq. j1_expanded) -> WENO-5 fluxes (App. A.2)
//   -> L[psi] (Eq. cast) -> Runge-Kutta combination.
//
// The state stores (phi_k, theta_k) of a cell as one pair, and the two
// components go through the same arithmetic, so every such step is written
// once on pairs: packed two-lane FP32 instructions in FP32, two scalar
// instructions in FP64.  Velocities are processed with their mirror images
// (the Gauss-Hermite set is symmetric, p_{Q-1-k} = -p_k).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "qlbm_internal.h"

namespace qlbm {

// ---------------------------------------------------------------------------
// Pairs of the working precision
template <typename Real>
struct PairOf;
template <>
struct PairOf<float> {
    using T = float2;
};
template <>
struct PairOf<double> {
    using T = double2;
};
template <typename Real>
using P2 = typename PairOf<Real>::T;

__device__ __forceinline__ float2 mk2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mk2(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float2 sp2(float a) { return make_float2(a, a); }
__device__ __forceinline__ double2 sp2(double a) { return make_double2(a, a); }

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b, one packed subtraction (PTX sub.rn.f32x2: no constant pair to hold
// in registers, unlike a fused multiply-add by -1, which rounds the same)
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;"
        : "=l"(r)
        : "l"(*reinterpret_cast<unsigned long long *>(&a)), "l"(*reinterpret_cast<unsigned long long *>(&b)));
    return *reinterpret_cast<float2 *>(&r);
}

__device__ __forceinline__ double2 add2(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 mul2(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ double2 fma2(double2 a, double2 b, double2 c)
{
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ double2 sub2(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// Precision-exact overloads: float arguments stay in FP32 (FP64 runs at a
// small fraction of the FP32 rate on this GPU).
__device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float max_(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double max_(double a, double b) { return fmax(a, b); }

template <typename Real>
__device__ __forceinline__ Real rsqrt_(Real x);
template <>
__device__ __forceinline__ float rsqrt_<float>(float x) { return rsqrtf(x); }
template <>
__device__ __forceinline__ double rsqrt_<double>(double x) { return rsqrt(x); }

template <typename Real>
__device__ __forceinline__ Real log_(Real x);
template <>
__device__ __forceinline__ float log_<float>(float x) { return logf(x); }
template <>
__device__ __forceinline__ double log_<double>(double x) { return log(x); }

template <typename Real>
__device__ __forceinline__ Real exp_(Real x);
template <>
__device__ __forceinline__ float exp_<float>(float x) { return expf(x); }
template <>
__device__ __forceinline__ double exp_<double>(double x) { return exp(x); }

template <typename Real>
__device__ __forceinline__ Real rcp_(Real x);
// FP32: the hardware reciprocal approximation alone (PTX rcp.approx.ftz.f32),
// for normal x; __fdividef(1, x) gives the same values for the arguments used
// here but adds a multiply and range checks to every reciprocal.
template <>
__device__ __forceinline__ float rcp_<float>(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
template <>
__device__ __forceinline__ double rcp_<double>(double x) { return 1.0 / x; }

// An exact power of two s with s x in [1, 4), for finite x >= 0 (s = 2^(e'-bias)
// where e' is the complement of x's exponent field with its lowest bit
// cleared; x = 0 gives a large finite s): one logic operation.
__device__ __forceinline__ float pow2_recip_(float x)
{
    return __uint_as_float(~__float_as_uint(x) & 0x7F000000u);
}
__device__ __forceinline__ double pow2_recip_(double x)
{
    return __hiloint2double(~__double2hiint(x) & 0x7FE00000, 0);
}

// max(a, b, c) of finite values (a single three-input max in FP32).
__device__ __forceinline__ float max3_(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ double max3_(double a, double b, double c) { return fmax(a, fmax(b, c)); }

// Smallest positive normal number of the working precision.
template <typename Real>
__device__ __forceinline__ Real min_normal_();
template <>
__device__ __forceinline__ float min_normal_<float>() { return 1.17549435e-38f; }
template <>
__device__ __forceinline__ double min_normal_<double>() { return 2.2250738585072014e-308; }

// ---------------------------------------------------------------------------
// Double-FP32 arithmetic: a value held as the unevaluated sum h + l of two
// floats, |l| <= ulp(h)/2 after normalisation, about 48 significant bits.
// two_sum is Knuth's error-free sum (no ordering needed), fast_two_sum Dekker's
// (|a| >= |b|), and products are made exact with one fma (Dekker/Knuth
// error-free transformations; the build never contracts a * b + c by itself).
struct FF {
    float h, l;
};
__device__ __forceinline__ FF two_sum(float a, float b)
{
    const float s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ FF fast_two_sum(float a, float b)
{
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ FF ff_add(FF a, FF b)
{
    const FF s = two_sum(a.h, b.h);
    return fast_two_sum(s.h, s.l + (a.l + b.l));
}
__device__ __forceinline__ FF ff_neg(FF a) { return {-a.h, -a.l}; }
// A double stored bit for bit in the two floats of an FF (h: high word, l: low
// word), so that FP64 and double-FP32 accumulators can share registers.
__device__ __forceinline__ double as_double(FF a)
{
    return __hiloint2double(__float_as_int(a.h), __float_as_int(a.l));
}
__device__ __forceinline__ FF as_ff(double d)
{
    return {__int_as_float(__double2hiint(d)), __int_as_float(__double2loint(d))};
}
__device__ __forceinline__ FF ff_mul(FF a, FF b)
{
    const float p = a.h * b.h;
    const float e = fmaf(a.h, b.h, -p);
    return fast_two_sum(p, fmaf(a.h, b.l, fmaf(a.l, b.h, e)));
}
__device__ __forceinline__ FF ff_mul_f(FF a, float b)
{
    const float p = a.h * b;
    return fast_two_sum(p, fmaf(a.l, b, fmaf(a.h, b, -p)));
}
// a / b: one quotient digit from an approximate reciprocal, then the exact
// remainder a - q b gives the correction digit.
__device__ __forceinline__ FF ff_div(FF a, FF b)
{
    const float r = __fdividef(1.0f, b.h);
    const float q = a.h * r;
    const float p = q * b.h;
    const float pe = fmaf(q, b.h, -p);
    const float rem = ((a.h - p) - pe) + fmaf(-q, b.l, a.l);
    return fast_two_sum(q, rem * r);
}

// ---------------------------------------------------------------------------
// WENO-5 value at the interface i+1/2 for a positive advection velocity
// (App. A.2), from f_{i-2..i+2}, for both components of the pairs.  Weights
// are delta_q / beta_q^2 normalised, with no epsilon; FP32 evaluates that
// quotient with reciprocals (below), FP64 in the product form
//   w_q = delta_q prod_{r != q} beta_r^2 / sum_s delta_s prod_{r != s} beta_r^2,
// equal to the quotient form wherever all beta_q > 0.  The indicators are
// first rescaled by one exact power of two (the weights depend only on their
// ratios).  Single-zero rows of Table weno_x come out of the product form;
// multi-zero rows give f0 (see below).  Candidates are differences from f0,
// so constant data give exactly f0.
template <typename Real>
__device__ __forceinline__ P2<Real> weno5_face2(P2<Real> fm2, P2<Real> fm1, P2<Real> f0, P2<Real> fp1, P2<Real> fp2)
{
    using V = P2<Real>;
    const V Dm2n = sub2(fm2, fm1);  // -(f_{i-1} - f_{i-2})
    const V Dm1 = sub2(f0, fm1);
    const V D0 = sub2(fp1, f0);
    const V D1 = sub2(fp2, fp1);
    // Indicators of Eq. (weno5_sigma) in the first differences a = f_{i-2} - f_{i-1}
    // (Dm2n), b = f_i - f_{i-1} (Dm1), b' = f_{i+1} - f_i (D0), c = f_{i+2} - f_{i+1} (D1):
    // 12 beta_q = 13 d_q^2 + 3 e_q^2 with the second differences d_q and the one-sided
    // differences e_q expands to 16 times
    //   a (a + 2.75 b) + 2.5 b^2,   b (b - 1.25 b') + b'^2,   c (c - 2.75 b') + 2.5 b'^2,
    // and the common factor 3/4 cancels in the weights.  Each form is positive definite
    // (its coefficient matrix has smallest eigenvalue 0.18 and 0.375), so it is zero only
    // where its differences are, and it is evaluated to a few units of rounding.
    const V Bsq = mul2(Dm1, Dm1), Bpsq = mul2(D0, D0);
    V b1 = fma2(sp2(Real(2.5)), Bsq, mul2(Dm2n, fma2(sp2(Real(2.75)), Dm1, Dm2n)));
    V b2 = fma2(Dm1, fma2(sp2(Real(-1.25)), D0, Dm1), Bpsq);
    V b3 = fma2(sp2(Real(2.5)), Bpsq, mul2(D1, fma2(sp2(Real(-2.75)), D0, D1)));
    // (delta_q / delta_1)(F^q - f0): candidates of Eq. (weno5_flux_x) relative to f0 with
    // the ideal weights of Eq. (weno5_delta), whose common factor delta_1 = 1/10 is
    // divided out of the numerator and the denominator of the face value
    const V D0x = add2(D0, D0);
    const V c1 = fma2(sp2(Real(1.0 / 3.0)), Dm2n, mul2(sp2(Real(5.0 / 6.0)), Dm1));
    const V c2 = add2(Dm1, D0x);
    const V c3 = fma2(sp2(Real(-0.5)), D1, D0x);
    const V sc = mk2(pow2_recip_(max3_(b1.x, b2.x, b3.x)), pow2_recip_(max3_(b1.y, b2.y, b3.y)));
    if constexpr (sizeof(Real) == 4) {
        // FP32: the quotient form itself, 1/beta_q^2 from the hardware reciprocal
        // (the special-function unit has room where the FMA pipes have none).  The
        // rescaled indicators lie in [0, 4), the largest in [1, 4); the same fused
        // multiply-add raises each by 2^-50, which bounds 1/beta^2 by 2^100 (the
        // numerator stays finite for differences below 2^26).  Nonzero FP32
        // indicators of one face differ from the largest by less than 2^54, so
        // the raise moves weight only between stencils flat to within 2^-25 of
        // the face's largest difference, whose candidates agree to that level.
        // A vanishing indicator gets 1/beta^2 = 2^100 against at most 1 for the
        // largest: one zero takes all the weight and two or three share it as
        // delta_q, the rows of Table weno_x.
        const V e50 = sp2(Real(8.8817841970012523e-16));
        b1 = fma2(b1, sc, e50);
        b2 = fma2(b2, sc, e50);
        b3 = fma2(b3, sc, e50);
        const V r1 = mk2(rcp_(b1.x), rcp_(b1.y)), r2 = mk2(rcp_(b2.x), rcp_(b2.y)), r3 = mk2(rcp_(b3.x), rcp_(b3.y));
        const V a1 = mul2(r1, r1), a2 = mul2(r2, r2), a3 = mul2(r3, r3);
        const V D = fma2(sp2(Real(3)), a3, fma2(sp2(Real(6)), a2, a1));
        const V num = fma2(a1, c1, fma2(a2, c2, mul2(a3, c3)));
        const V rD = mk2(rcp_(D.x), rcp_(D.y));
        return fma2(num, rD, f0);
    } else {
        b1 = mul2(b1, sc);
        b2 = mul2(b2, sc);
        b3 = mul2(b3, sc);
        const V s1 = mul2(b1, b1), s2 = mul2(b2, b2), s3 = mul2(b3, b3);
        const V P1 = mul2(s2, s3), P2v = mul2(s1, s3), P3 = mul2(s1, s2);
        const V D = fma2(sp2(Real(3)), P3, fma2(sp2(Real(6)), P2v, P1));
        const V num = fma2(P1, c1, fma2(P2v, c2, mul2(P3, c3)));
        // D = 0 only when two or three indicators vanish.  beta_q = 0 means the three
        // values of stencil q are equal, so two vanishing indicators make the union of
        // those stencils constant, the candidates that carry weight in Table weno_x
        // equal f0 there, and the face value is f0: num = 0 in that case too, and D is
        // raised to the smallest normal number so that its reciprocal stays finite
        // (a D below it would have no finite reciprocal either).
        const Real dmin = min_normal_<Real>();
        const V rD = mk2(rcp_(max_(D.x, dmin)), rcp_(max_(D.y, dmin)));
        return fma2(num, rD, f0);
    }
}

// Asks the TMA unit to bring `bytes` (a multiple of 16, 16-byte aligned
// address) of global memory into L2; no data reach the SM and nothing waits.
__device__ __forceinline__ void prefetch_l2_bulk(const void *p, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Shared-memory address of a generic pointer into shared memory.
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// mbarrier of a CTA (PTX mbarrier.*): initialised for one arriving thread;
// the TMA unit signals the bytes of its bulk copies against it.
__device__ __forceinline__ void mbar_init(uint64_t *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bulk copy (TMA, no tensor map) of `bytes` from global to shared memory,
// completion counted on `bar`; both addresses 16-byte aligned, bytes a
// multiple of 16.  The lines are marked first for eviction from L2: a staged
// row is read by its own tile and the halo of its neighbours, and leaving L2 to
// the psi^n rows prefetched for the velocity loop measured 0.7 % faster.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
        : "memory");
}
// Orders this thread's earlier generic-proxy accesses to shared memory before
// later async-proxy (TMA) writes to it.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Polls of the staging mbarrier before a CTA gives up (each try_wait may
// itself suspend the thread, measured at about 3.7 us, so the limit is about
// 0.25 s, against microseconds for a tile's copies); a give-up sets bit 1 of
// the error word and the tile is skipped.
constexpr uint32_t kMbarPolls = 1u << 16;

// 1: stage the tile's rows with TMA bulk copies; 0: with 16-byte loads.
#ifndef QL_STAGE_TMA
#define QL_STAGE_TMA 1
#endif

// Sixth-order central difference of App. A.3 (times dx), centred on s.
template <typename Real>
__device__ __forceinline__ Real cd6_(const Real *v, int s)
{
    return Real(1.0 / 60.0) * (v[s + 3] - v[s - 3]) + Real(-3.0 / 20.0) * (v[s + 2] - v[s - 2]) +
           Real(0.75) * (v[s + 1] - v[s - 1]);
}

// CTA shape: WARPS warps update 31 WARPS cells and stage 4 more on each side.
template <int WARPS>
struct TileShape {
    static constexpr int threads = 32 * WARPS;
    static constexpr int tile = 31 * WARPS;
    static constexpr int seg = tile + 2 * kHalo;
};

// Shared memory of one stage CTA: the staged rows, 6 per-cell arrays, 2 more
// for chi_RET-FM, and 3 pairs per velocity pair.  The equilibrium table rows
// G[k][l] are read from the constant bank (every lane of a warp reads the same
// entry), which leaves the shared memory to the staged rows.
template <typename Real, int Q, int WARPS, bool RET = false>
constexpr size_t stage_smem_bytes()
{
    constexpr int SEG = TileShape<WARPS>::seg;
    return sizeof(P2<Real>) * size_t(Q) * SEG + sizeof(Real) * ((RET ? 8 : 6) * size_t(SEG)) +
           sizeof(P2<Real>) * 3 * size_t(Q / 2);
}

// 1: the FP32 mode combines its per-cell conserved sums in FP64 instead of
// double-FP32 in every solver (StageArgs::sums64 selects it per solver).
#ifndef QL_F32_SUMS_FP64
#define QL_F32_SUMS_FP64 0
#endif

// 16-byte staging loads each thread keeps in flight.
#ifndef QL_STAGE_LOAD_UNROLL
#define QL_STAGE_LOAD_UNROLL 4
#endif
constexpr int kStageLoadUnroll = QL_STAGE_LOAD_UNROLL;

// Velocity pairs of the update loop per iteration.
#ifndef QL_VLOOP_UNROLL
#define QL_VLOOP_UNROLL 4
#endif
constexpr int kVelocityLoopUnroll = QL_VLOOP_UNROLL;

// Resident CTAs per SM the FP32 stage kernels are compiled for (8-warp tiles;
// the register budget follows from it).
#ifndef QL_STAGE_MINBLOCKS_F32
#define QL_STAGE_MINBLOCKS_F32 3
#endif

// ---------------------------------------------------------------------------
// One Runge-Kutta stage (STAGE 1..3), or L[psi] itself (STAGE 0), on the tile
// of cells i0 .. i0 + 31 WARPS - 1 of one 1D domain.  All threads of the CTA
// call it together; it uses dynamic shared memory from `smem`.  FP64 tiles may
// be shared by nparts CTAs, part `part` updating the velocity pairs
// [part H / nparts, (part + 1) H / nparts); each computes the tile's moments and
// per-cell coefficients itself.
template <typename Real, int Q, int STAGE, int WARPS, bool RET = false>
__device__ __forceinline__ void stage_tile(const StageArgs &a, const int64_t i0, unsigned char *smem_raw,
                                           uint64_t *mbar, uint32_t phase, int part = 0, int nparts = 1)
{
    using V = P2<Real>;
    constexpr TabView TV = tab_view(Q);
    constexpr int H = Q / 2;  // velocity k = H + j has p > 0, its mirror H - 1 - j has -p
    constexpr int THREADS = TileShape<WARPS>::threads;
    constexpr int SEG = TileShape<WARPS>::seg;
    static_assert(Q % 2 == 0, "symmetric velocity sets of even size");
    V *s_psi = reinterpret_cast<V *>(smem_raw);               // [Q][SEG] (phi, theta)
    Real *s_n = reinterpret_cast<Real *>(s_psi + Q * SEG);   // per staged cell
    Real *s_u = s_n + SEG;
    Real *s_T = s_u + SEG;
    Real *s_q = s_T + SEG;
    Real *s_lnn = s_q + SEG;
    Real *s_lnT = s_lnn + SEG;
    Real *s_lnchi = s_lnT + SEG;  // chi_RET-FM: nbar, then ln chi(nbar)
    Real *s_nout = s_lnchi + SEG; // chi_RET-FM: density of the output, per owned cell
    // per velocity pair j: (p, p), (p^2, p^2), (w dt p / dx, w dt p / dx)
    V *s_pt = reinterpret_cast<V *>(s_n + SEG * (RET ? 8 : 6));
    constexpr bool ret = RET;  // chi_RET-FM: a.nbar and a.nout are set
    // Runge-Kutta weight of v = psi + dt L in the stage output (c psi^n + w v):
    // 1, 1/4 and fl(2/3), whose complement 1 - w is exact (Sterbenz)
    const Real rk_w = STAGE == 2 ? Real(0.25) : (STAGE == 3 ? Real(2.0 / 3.0) : Real(1));

    const int t = threadIdx.x;
    const int64_t stride = a.stride;
    const V *__restrict__ in = static_cast<const V *>(a.in);

    // 1. Stage cells i0-kHalo .. i0+tile+kHalo-1 of every row: one thread has
    //    the TMA unit copy the Q row segments (SEG pairs each) while the others
    //    load the tables; or every thread copies 16-byte vectors.  Source rows
    //    start at pair r stride + i0: stride is even and i0 a multiple of 4, so
    //    with 16-byte aligned buffers every segment starts 16-byte aligned.
    {
        static_assert((SEG * sizeof(V)) % 16 == 0 && (TileShape<WARPS>::tile * sizeof(V)) % 16 == 0,
                      "TMA bulk copy alignment");
        if (QL_STAGE_TMA) {
            if (t == 0) {
                fence_proxy_async_smem();  // the previous tile's reads of s_psi come first
                mbar_arrive_expect_tx(mbar, uint32_t(Q * SEG * sizeof(V)));
                if (!a.fault)  // failure-detection tests: no copy is issued, the wait below gives up
                    for (int r = 0; r < Q; ++r)
                        bulk_copy_g2s(s_psi + r * SEG, in + r * stride + i0, uint32_t(SEG * sizeof(V)), mbar);
            }
        } else {
            constexpr int PPV = 16 / sizeof(V);  // pairs per vector
            constexpr int VPR = SEG / PPV;       // vectors per row
            static_assert(SEG % PPV == 0, "staging shape");
#pragma unroll kStageLoadUnroll
            for (int e = t; e < Q * VPR; e += THREADS) {
                const int r = e / VPR, vv = e - r * VPR;
                const uint4 v = __ldg(reinterpret_cast<const uint4 *>(in + r * stride + i0) + vv);
                reinterpret_cast<uint4 *>(s_psi + r * SEG)[vv] = v;
            }
        }
        if (t < H) {
            const Real p = QL_TAB[TV.p + H + t];
            const Real adv = STAGE == 0 ? Real(a.inv_dx) : Real(a.dt) * rk_w * Real(a.inv_dx);
            s_pt[3 * t] = sp2(p);
            s_pt[3 * t + 1] = sp2(QL_TAB[TV.p2 + H + t]);
            s_pt[3 * t + 2] = sp2(p * adv);
        }
        // nbar of staged cell c sits at column i0 + c (the buffer has a row stride of columns)
        if (ret)
            for (int c = t; c < SEG; c += THREADS) s_lnchi[c] = static_cast<const Real *>(a.nbar)[i0 + c];
    }
    if (QL_STAGE_TMA) {
        // every thread waits for the copies; the give-up decision is CTA-wide
        uint32_t polls = 0;
        while (!mbar_try_wait(mbar, phase) && ++polls < kMbarPolls) {
        }
        if (__syncthreads_or(polls >= kMbarPolls)) {
            if (t == 0) atomicOr(a.err, 2u);
            // let copies still in flight land before the shared memory is reused
            polls = 0;
            while (!mbar_try_wait(mbar, phase) && ++polls < kMbarPolls) {
            }
            __syncthreads();
            return;
        }
    } else {
        __syncthreads();
    }

    // 2. Moments of staged cell c (cell i0 - kHalo + c), Sec. II.D, from raw
    //    sums over velocity pairs.  FP64 mode sums in FP64.  FP32 mode sums
    //    groups of 8 pairs in FP32 and combines the groups' mass, momentum and
    //    energy sums either in FP64 (a.sums64) or in double-FP32 arithmetic,
    //    deriving u and T in the same arithmetic (FP64 runs at a small fraction
    //    of the FP32 rate on this GPU); the heat-flux sums stay in FP32.
    const bool kFF = sizeof(Real) == 4 && !QL_F32_SUMS_FP64 && !a.sums64;
    for (int c = t; c < SEG; c += THREADS) {
        constexpr int GRP = sizeof(Real) == 8 ? H : 8;
        // the FP64 sums (FP64 mode, or a.sums64) share the registers of the
        // double-FP32 ones: a double is held as its two 32-bit halves in (h, l)
        FF F0{0.f, 0.f}, F1{0.f, 0.f}, FE{0.f, 0.f};
        Real tS2 = 0, tS3 = 0, tR0 = 0, tR1 = 0;
#pragma unroll
        for (int g = 0; g < H; g += GRP) {
            V s01 = sp2(Real(0)), s11 = sp2(Real(0));  // (S0, R0), (S1, R1) partials
            Real s2 = 0, s3 = 0;
#pragma unroll
            for (int j = g; j < g + GRP && j < H; ++j) {
                const Real p = QL_TAB[TV.p + H + j];
                const V fa = s_psi[(H + j) * SEG + c], fb = s_psi[(H - 1 - j) * SEG + c];
                const V sm = add2(fa, fb), df = sub2(fa, fb);
                s01 = add2(s01, sm);
                s11 = fma2(sp2(p), df, s11);
                s2 = fma_(QL_TAB[TV.p2 + H + j], sm.x, s2);
                s3 = fma_(QL_TAB[TV.p3 + H + j], df.x, s3);
            }
            if (kFF) {
                // error-free accumulation: h takes the rounded sum, l its errors
                const FF a0 = two_sum(F0.h, float(s01.x)), a1 = two_sum(F1.h, float(s11.x));
                const FF a2 = two_sum(FE.h, float(s2)), a3 = two_sum(a2.h, float(s01.y));
                F0 = {a0.h, F0.l + a0.l};
                F1 = {a1.h, F1.l + a1.l};
                FE = {a3.h, FE.l + (a2.l + a3.l)};
            } else {
                F0 = as_ff(as_double(F0) + double(s01.x));
                F1 = as_ff(as_double(F1) + double(s11.x));
                FE = as_ff(as_double(FE) + double(s2 + s01.y));
            }
            tS2 += s2;
            tS3 += s3;
            tR0 += s01.y;
            tR1 += s11.y;
        }
        // 3 n T = sum xi^2 phi + sum theta = (S2 + R0) - u S1
        Real uf, Tf, nf;
        if (kFF) {
            const FF n = fast_two_sum(F0.h, F0.l), m1 = fast_two_sum(F1.h, F1.l), me = fast_two_sum(FE.h, FE.l);
            const FF u = ff_div(m1, n);
            const FF T = ff_div(ff_add(me, ff_neg(ff_mul(u, m1))), ff_mul_f(n, 3.0f));
            nf = Real(n.h);
            uf = Real(u.h);
            Tf = Real(T.h);
        } else {
            // 1/n from a working-precision reciprocal refined by Newton steps in FP64
            // (one step gives ~1e-14 after an FP32 seed, two after FP64's own division)
            const double n = as_double(F0), M1 = as_double(F1), ME = as_double(FE);
            double rn = double(rcp_(Real(n)));
            rn = fma(rn, fma(-n, rn, 1.0), rn);
            if (sizeof(Real) == 8) rn = fma(rn, fma(-n, rn, 1.0), rn);
            const double u = M1 * rn;
            const double T = fma(-u, M1, ME) * rn * (1.0 / 3.0);
            uf = Real(u);
            Tf = Real(T);
            nf = Real(n);
        }
        // 2 q = sum xi^3 phi + sum xi theta = S3 + R1 - u (3 S2 + R0) + 2 u^2 S1
        const Real q = Real(0.5) * (tS3 + tR1 - uf * fma_(Real(3), tS2, tR0) + Real(2) * uf * uf * (uf * nf));
        const int64_t i = i0 - kHalo + c;
        if (i >= 0 && i < a.nx) {
            if (!(nf > Real(0)) || !(Tf > Real(0)) || !isfinite(uf) || !isfinite(q) || !isfinite(nf) || !isfinite(Tf))
                atomicOr(a.err, 1u);
        }
        s_n[c] = nf;
        s_u[c] = uf;
        s_T[c] = Tf;
        s_q[c] = q;
        s_lnn[c] = log_(nf);
        s_lnT[c] = log_(Tf);
        if (ret) {
            // Eq. (chi_ret): chi_SET of the averaged density
            const Real eb = Real(a.eta0) * s_lnchi[c] * Real(a.inv_rho_ref), omb = Real(1) - eb;
            s_lnchi[c] = log_(Real(0.5) * (Real(2) - eb) / (omb * omb * omb));
        }
    }
    __syncthreads();

    // 3. Update.  Lane l of warp w handles staged cell s = 31 w + l + 3: it
    //    computes the interface values on the right face of s, and (l >= 1)
    //    updates cell s, whose left-face values come from lane l-1.
    const int lane = t & 31, warp = t >> 5;
    const int s = 31 * warp + lane + 3;
    const int64_t i = i0 - kHalo + s;
    const bool owner = lane != 0 && i < a.nx;

    const Real n = s_n[s], u = s_u[s], T = s_T[s], q = s_q[s];
    const Real inv_dx = Real(a.inv_dx);
    const Real dlnn = cd6_(s_lnn, s) * inv_dx;
    const Real du = cd6_(s_u, s) * inv_dx;
    const Real dlnT = cd6_(s_lnT, s) * inv_dx;

    // Secs. II.A-B: eta, chi_SET, Y = b rho chi, tau = mu / P_i, Pr.
    const Real rhat = n * Real(a.inv_rho_ref);
    const Real eta = Real(a.eta0) * rhat;
    const Real ome = Real(1) - eta;
    const Real rome = rcp_(ome);
    const Real chi = ret ? exp_(s_lnchi[s]) : Real(0.5) * (Real(2) - eta) * (rome * rome * rome);
    const Real Y = Real(4) * eta * chi;
    const Real muf = fma_(fma_(Real(0.16 * (1.0 + 12.0 / 3.14159265358979323846)), Y, Real(0.8)), Y, Real(1));
    const Real sqT = T * rsqrt_(T);
    const Real inv_tau = rhat * chi * sqT * rcp_(Real(a.tau_pref) * muf);
    Real Pr = Real(a.pr_const);
    if (a.pr_mode) {
        const Real laf =
            fma_(fma_(Real(0.36 * (1.0 + 32.0 / (9.0 * 3.14159265358979323846))), Y, Real(1.2)), Y, Real(1));
        Pr = Real(2.0 / 3.0) * muf * rcp_(laf);
    }
    const Real invT = rcp_(T);
    // Shakhov: A = (1 - Pr) q / (5 P_i T), P_i = n T
    const Real A = (Real(1) - Pr) * q * invT * invT * (Real(0.2) * rcp_(n));
    const Real Yj = a.enskog ? Y : Real(0);
    // chi_SET: d ln chi = eta (3/(1-eta) - 1/(2-eta)) d ln rho (chi depends on the local eta only);
    // chi_RET-FM: 6th-order difference of ln chi(nbar)
    const Real dlnchi =
        ret ? cd6_(s_lnchi, s) * inv_dx : eta * (Real(3) * rome - rcp_(Real(2) - eta)) * dlnn;
    const Real G = dlnchi + Real(2) * dlnn;
    // Targets over the equilibrium, cubic in xi = p_k - u:
    //   phi:   (1/tau)(1 + A xi (xi^2/T - 3)) - Y [xi G + 3/5 (xi^2/T - 1) du + 3/10 (xi^3/T + xi/3) dlnT]
    //   theta: (1/tau)(1 + A xi (xi^2/T - 1)) - Y [xi G + 3/5 (xi^2/T - 1/3) du + 3/10 (xi^3/T + 7 xi/3) dlnT]
    // times n g_k and 2 T n g_k; the pairs below hold (phi, theta) coefficients
    // already multiplied by n and 2 T n.
    const Real a0 = fma_(Real(0.6) * Yj, du, inv_tau);
    const Real a1 = -Real(3) * A * inv_tau - Yj * G - Real(0.1) * Yj * dlnT;
    const Real a2 = -Real(0.6) * Yj * du * invT;
    const Real a3 = (A * inv_tau - Real(0.3) * Yj * dlnT) * invT;
    const Real b0 = fma_(Real(0.2) * Yj, du, inv_tau);
    const Real b1 = -A * inv_tau - Yj * G - Real(0.7) * Yj * dlnT;
    // Stages 1-3 fold dt and the Runge-Kutta weight of v into the targets (see
    // the velocity loop).
    const Real ndt = STAGE == 0 ? n : n * (Real(a.dt) * rk_w);
    const Real nphi = ndt, nth = Real(2) * T * ndt;
    const V C0 = mk2(a0 * nphi, b0 * nth), C1 = mk2(a1 * nphi, b1 * nth);
    const V C2 = mk2(a2 * nphi, a2 * nth), C3 = mk2(a3 * nphi, a3 * nth);
    // The same cubic as a polynomial in y = xi + u = +-p (Taylor shift by -u,
    // Horner's scheme): P(+-p) = E(p^2) +- p O(p^2) with E = D0 + D2 p^2 and
    // O = D1 + D3 p^2, so both velocities of a pair share E and O.
    V D0 = C0, D1 = C1, D2 = C2;
    const V D3 = C3;
    {
        const V mu = sp2(-u);
        D2 = fma2(mu, D3, D2);
        D1 = fma2(mu, D2, D1);
        D0 = fma2(mu, D1, D0);
        D2 = fma2(mu, D3, D2);
        D1 = fma2(mu, D2, D1);
        D2 = fma2(mu, D3, D2);
    }

    // Hermite coefficients of the equilibrium, Eq. (g_alpha), scaled as
    // d_l = l! c_l: d_0 = 1, d_1 = u, d_l = u d_{l-1} + (l-1)(T-1) d_{l-2} (the
    // factor l - 1 from the table; its equilibrium rows carry the 1/l!), held as
    // pairs (d_{2m}, d_{2m+1}).
    V ch[H];
    {
        Real cm2 = Real(1), cm1 = u;
        ch[0] = mk2(cm2, cm1);
        const Real Tm1 = T - Real(1);
#pragma unroll
        for (int m = 1; m < H; ++m) {
            const Real ce = fma_(u, cm1, (QL_TAB[TV.cb + 2 * m] * Tm1) * cm2);
            const Real co = fma_(u, ce, (QL_TAB[TV.cb + 2 * m + 1] * Tm1) * cm1);
            ch[m] = mk2(ce, co);
            cm2 = ce;
            cm1 = co;
        }
    }

    // STAGE 0: L[psi] = target - psi / tau - advection.  Stages 1-3 form
    // w v = w (psi + dt L[psi]) directly as w (1 - dt/tau) psi + w dt target -
    // w dt advection (targets and the advection table already scaled by w dt).
    const Real dt = Real(a.dt);
    const V kpsi = sp2(STAGE == 0 ? -inv_tau : rk_w * (Real(1) - dt * inv_tau));
    const V *__restrict__ base = static_cast<const V *>(a.base);
    V *out = static_cast<V *>(a.out);
    const int64_t col = kHalo + i;
    // velocity pairs of this CTA (all of them in FP32)
    const int j0 = sizeof(Real) == 8 ? (part * H) / nparts : 0;
    const int j1 = sizeof(Real) == 8 ? ((part + 1) * H) / nparts : H;
    // chi_RET-FM: the output density of the owned cell, summed over the velocity
    // loop (only this thread touches s_nout[s]); a CTA with part of the
    // velocities leaves it to a density pass after the stage
    const bool own_density = RET && STAGE != 0 && (sizeof(Real) == 4 || nparts == 1);
    if (own_density && owner) s_nout[s] = Real(0);

    // psi^n rows of the tile's cells (columns kHalo + i0 .. kHalo + i0 + tile - 1,
    // inside every row, whose stride leaves room for the staged segment): before
    // the velocity loop one thread asks the TMA unit to bring all of them into
    // L2 (2 Q x tile pairs, 64 KB per CTA in FP32), so the loads of psi^n in the
    // loop hit L2.  Byte offsets are multiples of 16: stride is even, kHalo + i0
    // a multiple of 4 pairs, tile x sizeof(V) a multiple of 16.
    constexpr uint32_t kRowBytes = uint32_t(TileShape<WARPS>::tile * sizeof(V));
    static_assert(kRowBytes % 16 == 0, "bulk prefetch size");
    if (STAGE >= 2 && t == 0)
        for (int r = 0; r < Q; ++r) prefetch_l2_bulk(base + int64_t(r) * stride + kHalo + i0, kRowBytes);

    // FP32 stage 1 runs faster with the loop rolled (0.625 -> 0.609 ms per launch on the Sod tube, 2^22 cells,
    // Q = 32), stages 2-3 with kVelocityLoopUnroll pairs per iteration (rolled: 0.682 -> 0.697 ms)
    constexpr int kUnroll = (STAGE == 1 && sizeof(Real) == 4) ? 1 : kVelocityLoopUnroll;
#pragma unroll kUnroll
    for (int j = j0; j < j1; ++j) {
        const int kp = H + j, km = H - 1 - j;

        const int64_t ip = int64_t(kp) * stride + col, im = int64_t(km) * stride + col;
        // psi^n of this cell, loaded before the arithmetic that hides its latency
        // (every lane's column lies inside the row: ghost or padding columns at worst)
        V bp = sp2(Real(0)), bm = sp2(Real(0));
        if (STAGE >= 2) {
            bp = base[ip];
            bm = base[im];
        }
        // (p, p), (p^2, p^2), (w dt p / dx, w dt p / dx) of this pair (p / dx for STAGE 0)
        const V *pt = s_pt + 3 * j;
        const V *rp = s_psi + kp * SEG;
        const V *rm = s_psi + km * SEG;
        // WENO-5 values at the right face of s: upwind stencil for +p, mirrored for -p
        const V fp0 = rp[s], fm0 = rm[s];
        const V hp = weno5_face2<Real>(rp[s - 2], rp[s - 1], fp0, rp[s + 1], rp[s + 2]);
        const V hm = weno5_face2<Real>(rm[s + 3], rm[s + 2], rm[s + 1], fm0, rm[s - 1]);
        const V hpl = mk2(__shfl_up_sync(0xffffffffu, hp.x, 1), __shfl_up_sync(0xffffffffu, hp.y, 1));
        const V hml = mk2(__shfl_up_sync(0xffffffffu, hm.x, 1), __shfl_up_sync(0xffffffffu, hm.y, 1));

        // g at +p and -p: even and odd Hermite parts, h_l(-p) = (-1)^l h_l(p); the
        // table row of p_k (k = H + j) from the constant bank
        V eo = sp2(Real(0));
        const V *Gj = reinterpret_cast<const V *>(&QL_TAB[TV.G + (H + j) * Q]);
#pragma unroll
        for (int m = 0; m < H; ++m) eo = fma2(Gj[m], ch[m], eo);
        const Real gpv = eo.x + eo.y, gmv = eo.x - eo.y;

        // targets, Eq. (cast): L[psi] = target - psi / tau - (p/dx)(h - h_left) for
        // STAGE 0, w v = w (psi + dt L[psi]) for stages 1-3
        const V E = fma2(D2, pt[1], D0);
        const V O = mul2(fma2(D3, pt[1], D1), pt[0]);
        const V Pp = add2(E, O), Pm = sub2(E, O);
        const V vp = fma2(pt[2], sub2(hpl, hp), fma2(fp0, kpsi, mul2(sp2(gpv), Pp)));
        const V vm = fma2(pt[2], sub2(hm, hml), fma2(fm0, kpsi, mul2(sp2(gmv), Pm)));

        if (owner) {
            V op = vp, om = vm;
            if (STAGE >= 2) {
                // c psi^n + w v with (c, w) = (3/4, 1/4) and (1 - fl(2/3), fl(2/3)):
                // the two weights sum to exactly one in any precision (1/3 and 2/3
                // both rounded to FP32 sum to 1 + 4e-8, a per-step bias)
                const V c = sp2(Real(1) - rk_w);
                op = fma2(c, bp, vp);
                om = fma2(c, bm, vm);
            }
            // streaming stores: the next stage reads them from memory, not from L2
            __stcs(out + ip, op);
            __stcs(out + im, om);
            if (own_density) s_nout[s] += op.x + om.x;
        }
    }
    if (STAGE != 0 && a.periodic && owner && (i < kHalo || i >= a.nx - kHalo)) {
        // periodic images in the ghost columns of the other end: this thread
        // copies the rows it has just written in the column (its own stores, read back)
        for (int k = H - j1; k < H + j1; ++k) {
            if (k >= H - j0 && k < H + j0) continue;  // rows of the other CTAs of the tile
            const V v = out[int64_t(k) * stride + col];
            if (i < kHalo) out[int64_t(k) * stride + col + a.nx] = v;
            if (i >= a.nx - kHalo) out[int64_t(k) * stride + col - a.nx] = v;
        }
    }
    if (own_density && owner) static_cast<Real *>(a.nout)[i] = s_nout[s];
}

// FP32: QL_STAGE_MINBLOCKS_F32 CTAs per SM up to Q = 32; Q = 40 holds twice the
// Hermite coefficients and 80 KB of staged rows, and runs 2 CTAs per SM.
template <typename Real, int Q>
struct StageOccupancy {
    static constexpr int value = sizeof(Real) == 4 ? (Q > 32 ? 2 : QL_STAGE_MINBLOCKS_F32) : 1;
};

// One Runge-Kutta stage over a whole domain: CTA b updates tile b, or in FP64
// with a.vsplit > 1 the velocity range b % vsplit of tile b / vsplit.
template <typename Real, int Q, int STAGE, bool RET>
__global__ void __launch_bounds__(kThreads, StageOccupancy<Real, Q>::value) fdlb_stage_kernel(StageArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar;
    if (QL_STAGE_TMA) {
        if (threadIdx.x == 0) mbar_init(&mbar);
        __syncthreads();
    }
    // Programmatic dependent launch (the solver launches its stages that way):
    // the next stage may be scheduled once every CTA of this one has started,
    // and this one reads or writes no state before the previous kernel in the
    // stream has completed (a no-op for plain launches).  Each stage waits for
    // its predecessor, so a stage's start implies that all earlier ones ended.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int vs = sizeof(Real) == 8 ? a.vsplit : 1;
    const int64_t tile = int64_t(blockIdx.x) / vs;
    const int part = int(int64_t(blockIdx.x) - tile * vs);
    stage_tile<Real, Q, STAGE, kWarps, RET>(a, tile * kTile, smem_raw, &mbar, 0u, part, vs);
}

// ---------------------------------------------------------------------------
// A run of steps in one launch (FP32, chi_SET).  With one launch per stage,
// each stage waits for the slowest CTA of the one before, and its first wave
// of CTAs stages its tiles all at once.  Here CTA b of the launch takes ticket
// b, tile b mod N of stage b / N of the run (N tiles), and starts as soon as
// the previous stage of the tiles it reads has completed, so consecutive
// stages overlap.
//
// Dependencies of stage g of tile i: stage g - 1 of tiles i - 1, i and i + 1
// (modulo N with a periodic boundary; there tiles 0 and N - 2 also depend on
// each other, because when the last tile holds fewer cells than the halo, tile
// N - 2 stages ghost images that tile 0 writes and writes some that tile 0
// stages).  Overwrites are ordered by the same chain: whoever read a buffer's
// cells at stage g - 1 is a tile that the writer at stage g waits for, and
// readers at earlier stages completed before those.
//
// Ordering: a tile's stores (all threads, then a CTA barrier) are published by
// thread 0 as the tile's count of completed stages (counted from the solver's
// first run), a release store at GPU scope.  A consumer's thread 0 reads the counts with acquire loads, then
// orders its staging copies (async proxy) after them; its other threads read
// after CTA barriers.
//
// Progress: a ticket's dependencies hold smaller tickets, that is CTAs of
// smaller index, which the hardware starts first (one-dimensional grids are
// dispatched in index order, the assumption single-pass scans with
// look-back also make), so the smallest unfinished ticket always has what it
// needs.  Waits are bounded all the same: a CTA that gives up sets bit 2 of
// the error word and returns, and every CTA that finds the bit while waiting
// returns too (the state is then invalid and the host reports the error).
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Orders this thread's earlier generic-proxy view of global memory before its
// later async-proxy (TMA) reads.
__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// True once stage g - 1 of every tile that stage g of `tile` reads has
// completed (always for the run's first stage).
// Counts are kept modulo 2^32: count c has reached stage s when the signed
// difference c - s is not negative.
__device__ __forceinline__ bool reached_(unsigned c, unsigned s) { return int(c - s) >= 0; }
__device__ __forceinline__ bool run_ready(const unsigned *d, unsigned N, bool per, unsigned tile, unsigned g,
                                          unsigned g0)
{
    if (g == 0) return true;  // every tile completed the previous run
    const unsigned s = g0 + g;
    bool ok = reached_(ld_acquire_gpu(d + tile), s);
    if (tile > 0)
        ok &= reached_(ld_acquire_gpu(d + tile - 1), s);
    else if (per)
        ok &= reached_(ld_acquire_gpu(d + N - 1), s);
    if (tile + 1 < N)
        ok &= reached_(ld_acquire_gpu(d + tile + 1), s);
    else if (per)
        ok &= reached_(ld_acquire_gpu(d), s);
    if (per && N > 2) {
        if (tile == 0) ok &= reached_(ld_acquire_gpu(d + N - 2), s);
        if (tile == N - 2) ok &= reached_(ld_acquire_gpu(d), s);
    }
    return ok;
}

// Polls of a tile's dependencies before a CTA gives up (each poll is a round
// trip to L2 and a short sleep: about a second in all, against microseconds
// for a tile's stage).
constexpr uint32_t kRunPolls = 1u << 20;

template <int Q>
__global__ void __launch_bounds__(kThreads, StageOccupancy<float, Q>::value) fdlb_run_kernel(RunArgs r)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ int s_stop;
    __shared__ unsigned s_tile, s_count;  // read back by thread 0 after the tile
    // Programmatic dependent launch, as for the stage kernels: the next kernel
    // may be scheduled once every CTA of this one has started, and no CTA
    // touches the state before the previous kernel in the stream has completed.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int t = threadIdx.x;
    // fewer than 2^31 tickets per launch
    const unsigned N = unsigned(r.ntiles);
    const unsigned g = blockIdx.x / N;
    const unsigned tile = blockIdx.x - g * N;
    if (t == 0) {
        s_tile = tile;
        s_count = r.g0 + g + 1u;
        bool ok = run_ready(r.done, N, r.st[0][0].periodic != 0, tile, g, r.g0);
        for (uint32_t polls = 0; !ok;) {
            if (++polls >= kRunPolls || (*reinterpret_cast<volatile unsigned *>(r.st[0][0].err) & 4u)) {
                atomicOr(r.st[0][0].err, 4u);
                break;
            }
            __nanosleep(64);
            ok = run_ready(r.done, N, r.st[0][0].periodic != 0, tile, g, r.g0);
        }
        s_stop = !ok;
        if (ok) fence_proxy_async_global();
        if (QL_STAGE_TMA) mbar_init(&mbar);
    }
    __syncthreads();
    if (s_stop) return;
    const int64_t i0 = int64_t(tile) * kTile;
    // step g / 3 reads psi^n from buf0 (even steps) or buf1 (odd steps)
    const int k = int(g % 3u), odd = int((g / 3u) & 1u);
    if (k == 0) {
        stage_tile<float, Q, 1, kWarps, false>(r.st[odd][0], i0, smem_raw, &mbar, 0u);
    } else if (k == 1) {
        stage_tile<float, Q, 2, kWarps, false>(r.st[odd][1], i0, smem_raw, &mbar, 0u);
    } else {
        stage_tile<float, Q, 3, kWarps, false>(r.st[odd][2], i0, smem_raw, &mbar, 0u);
    }
    __syncthreads();  // every store of the tile is issued
    if (t == 0) st_release_gpu(r.done + s_tile, s_count);  // cumulative: orders the CTA's stores before it
}

// Batched form: per Runge-Kutta stage, one persistent launch per velocity set
// over the work list of (instance, tile) items of the instances with that Q
// (independent domains with their own size and gas parameters).  Each CTA
// walks the list with stride gridDim.x.
template <int WARPS>
struct BatchOccupancy {
    static constexpr int value = WARPS == 8 ? QL_STAGE_MINBLOCKS_F32 : 2 * QL_STAGE_MINBLOCKS_F32 - 1;
};

template <typename Real, int Q, int STAGE, int WARPS, bool RET = false>
__global__ void __launch_bounds__(32 * WARPS, sizeof(Real) == 4 ? BatchOccupancy<WARPS>::value : 1)
    fdlb_batch_stage_kernel(BatchArgs b)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar;
    if (QL_STAGE_TMA) {
        if (threadIdx.x == 0) mbar_init(&mbar);
        __syncthreads();
    }
    // The item's arguments live in shared memory and are read where they are used:
    // held in registers across the tile they pushed the Q = 24 and 32 kernels into
    // 100 - 150 bytes of spills (55.0 -> 57.5 G updates/s when moved here).
    __shared__ StageArgs s_args;
    uint32_t phase = 0;  // parity of the staging mbarrier, one phase per item
    for (int64_t w = blockIdx.x; w < b.nwork; w += gridDim.x, phase ^= 1u) {
        const int2 it = b.work[w];
        if (threadIdx.x == 0) {
            const BatchInstance &I = b.inst[it.x];
            StageArgs a;
            const int64_t off = I.off;
            const P2<Real> *A = static_cast<const P2<Real> *>(b.arena[0]) + off;
            const P2<Real> *Bb = static_cast<const P2<Real> *>(b.arena[1]) + off;
            const P2<Real> *C = static_cast<const P2<Real> *>(b.arena[2]) + off;
            // psi^(n+1) goes to the buffer of psi^(1), not in place (the host swaps
            // the first two buffers after each step)
            a.in = STAGE == 1 ? A : (STAGE == 2 ? Bb : C);
            a.base = A;
            a.out = const_cast<P2<Real> *>(STAGE == 2 ? C : Bb);
            a.nx = I.nx;
            a.stride = I.stride;
            a.inv_dx = I.inv_dx;
            a.dt = I.dt;
            a.eta0 = I.eta0;
            a.inv_rho_ref = I.inv_rho_ref;
            a.tau_pref = I.tau_pref;
            a.pr_const = I.pr_const;
            a.pr_mode = I.pr_mode;
            a.enskog = I.enskog;
            a.periodic = I.periodic;
            a.fault = 0;
            a.sums64 = b.sums64;
            a.vsplit = 1;
            a.err = b.err + it.x;
            // chi_RET-FM lists: the instance's nbar, and the densities of this stage's output
            a.nbar = RET ? static_cast<void *>(static_cast<Real *>(b.nbar) + I.noff) : nullptr;
            a.nout = RET ? static_cast<void *>(static_cast<Real *>(b.n) + I.noff) : nullptr;
            s_args = a;
        }
        __syncthreads();
        const int64_t i0 = int64_t(it.y) * TileShape<WARPS>::tile;
        stage_tile<Real, Q, STAGE, WARPS, RET>(s_args, i0, smem_raw, &mbar, phase);  // every item of this list has this Q
        __syncthreads();  // shared memory (and s_args) is reused by the next item
    }
}

}  // namespace qlbm
