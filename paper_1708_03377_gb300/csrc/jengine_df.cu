// FP64-accurate J-engine on the FP32 pipes: float-float ("df64") arithmetic.
//
// A df64 value is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2 (48-bit
// significand, FP32 exponent range).  Sums use Knuth's error-free two-sum, products the FMA
// two-product (Dekker 1971; the double-double scheme of Hida, Li and Bailey, 2001), so every
// operation is a handful of FP32 instructions: GB300 issues FP32 at ~70x its FP64 rate, which is
// what makes this faster than native DFMA for the fused McMurchie-Davidson contraction.
//
// Same work decomposition and normalisation as the FP64 core (one warp = 32 bra primitive pairs of
// class L_P, in exponent order, against the ket pairs of class L_Q <= L_P of the partner fragment),
// same screening, same outputs (FP64 Hermite fields pp_Jh):
//   * centres, exponents, sqrt(p), the weights u = p^{-1/2} D_P and the Boys table are df64 copies
//     of the FP64 data;
//   * beyond the asymptotic switch (T >= 36, warp-uniform in the common case) the unit-normalised
//     Hermite base is that of two point multipoles, (-1)^n (2n-1)!! / R^{2n+1}, one df64 reciprocal
//     square root per quartet (float seed + Newton steps); below it F_m comes from the same
//     grid-Taylor table (order 6, h = 0.05) evaluated in df64;
//   * R recursion and both contractions in df64; the bra field is flushed into FP64 registers
//     every 32 kets and scaled by (sqrt(pi)/2) p^{-1/2} at the end, the ket field is summed over the
//     warp in df64, scaled by (sqrt(pi)/2) q^{-1/2} in FP64 and added with one FP64 atomic
//     (floats converted by exponent re-biasing on the integer pipe).
// Values below the FP32 normal range (~1e-38) are flushed to zero, far below every tolerance.
// Classes with L_P >= 3 (d shells) and L_P + L_Q >= 5 use the native FP64 kernels.
#include <algorithm>
#include <climits>

#include "common.cuh"
#include "df64.cuh"
#include "internal.hpp"

namespace fef {

namespace {

using namespace ffa;

__device__ __forceinline__ df64 ld_df(const float2* p)
{
    const float2 v = __ldg(p);
    return df64(v.x, v.y);
}

constexpr float kSqrtPiHalfHi = (float)kSqrtPiHalf;
constexpr float kSqrtPiHalfLo = (float)(kSqrtPiHalf - (double)(float)kSqrtPiHalf);

// F_0..F_L at T in df64 from the df64 copy of the grid-Taylor table (row kidx from an FP32 T).
template <int L>
__device__ __forceinline__ void boys_df(const float2* __restrict__ table, df64 T, int kidx, df64* F)
{
    if (kidx < kBoysRows - 1) {
        const float2* row = table + (size_t)kidx * kBoysRowLen;
        const df64 d = ld_df(row + kBoysOrder + 1) - T;
#pragma unroll
        for (int m = 0; m <= L; ++m) {
            const float2* c = row + m * kBoysBlock;
            const float4 c01 = __ldg(reinterpret_cast<const float4*>(c));
            const float4 c23 = __ldg(reinterpret_cast<const float4*>(c + 2));
            const float4 c45 = __ldg(reinterpret_cast<const float4*>(c + 4));
            const float2 c6 = __ldg(c + 6);
            df64 f = fma(d, df64(c6.x, c6.y), df64(c45.z, c45.w));
            f = fma(d, f, df64(c45.x, c45.y));
            f = fma(d, f, df64(c23.z, c23.w));
            f = fma(d, f, df64(c23.x, c23.y));
            f = fma(d, f, df64(c01.z, c01.w));
            F[m] = fma(d, f, df64(c01.x, c01.y));
        }
    } else {
        const df64 r = rsqrt_df(T);
        const df64 half_inv_T = df64(0.5f, 0.0f) * (r * r);
        F[0] = df64(kSqrtPiHalfHi, kSqrtPiHalfLo) * r;
#pragma unroll
        for (int m = 1; m <= L; ++m) F[m] = F[m - 1] * (half_inv_T * df64(2 * m - 1));
    }
}

constexpr int kFlushKets = 32;

// The ket-side field is staged per warp (as in the FP64 core): lane l writes its float-float partial
// sums of up to 32 ket components into row l of a 32 x 33 shared-memory block; once the batch is
// full, the lane owning a slot sums its column in float-float and adds it to global memory.
constexpr int kDfBufLd = 33;
constexpr int kDfBufWarp = 32 * kDfBufLd;
struct DfKetBuf {
    float2* v;  // [32 lanes][kDfBufLd] (hi, lo)
    int* k;     // [32] ket pair of each batch position
};

template <int NQ>
__device__ __forceinline__ void df_ketbuf_flush(const DfKetBuf& kb, int cnt, double* __restrict__ QJ, size_t nQ,
                                                const double* __restrict__ rq, int lane)
{
    __syncwarp();
    if (lane < cnt * NQ) {
        df64 sum(0.0f, 0.0f);
#pragma unroll 4
        for (int r = 0; r < 32; ++r) {
            const float2 v = kb.v[r * kDfBufLd + lane];
            sum = sum + df64(v.x, v.y);
        }
        const int k = kb.k[lane / NQ];
        atomicAdd(QJ + (size_t)(lane % NQ) * nQ + k, (f2d(sum.hi) + f2d(sum.lo)) * (kSqrtPiHalf * __ldg(rq + k)));
    }
    __syncwarp();
}

// 1/sqrt(x) of a df64 x > 0 from a float seed s ~ x.hi^{-1/2} (relative error <= 2^-22): one float
// Newton step, then one df64 correction y = r + r e / 2 with e = 1 - x r^2 formed exactly enough
// (r^2 as an exact float product pair, 1 - (x r^2).hi exact by Sterbenz); relative error ~1e-14.
__device__ __forceinline__ df64 rsqrt_df_seed(df64 x, float s)
{
    const float r = s * fmaf(-0.5f * x.hi * s, s, 1.5f);
    const float rr = __fmul_rn(r, r);
    const df64 r2(rr, __fmaf_rn(r, r, -rr));
    const df64 p = x * r2;
    const float e = __fsub_rn(__fsub_rn(1.0f, p.hi), p.lo);
    return quick_two_sum(r, 0.5f * r * e);
}

// a * b for a df64 a and a float b
__device__ __forceinline__ df64 mul_df_f(df64 a, float b)
{
    const float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    return quick_two_sum(p, e);
}

// Unit-normalised Hermite base below the asymptotic switch (the FP64 core's convention):
// (2/sqrt(pi)) sqrt(alpha) F_n(T) (-2 alpha)^n with alpha = p q / (p + q), T = alpha R^2 and
// sqrt(alpha) = sqrt(p) sqrt(q) (p + q)^{-1/2}, in df64.  Out of line, so that the asymptotic path of
// the quartet loop carries none of its instructions.
template <int L>
struct BaseDf {
    df64 v[L + 1];
};
template <int L>
__device__ __noinline__ BaseDf<L> df_table_base(const float2* __restrict__ table, df64 p, df64 q, df64 sqp, df64 sqq,
                                                df64 R2, float Tf)
{
    BaseDf<L> b;
    const df64 s = p + q;
    const df64 r = rsqrt_df_seed(s, rsqrt_approx(s.hi));
    const df64 alpha = (p * q) * (r * r);
    df64 F[L + 1];
    boys_df<L>(table, alpha * R2, boys_row(Tf), F);
    df64 pre = df64(kTwoOverSqrtPiHi, kTwoOverSqrtPiLo) * ((sqp * sqq) * r);
    const df64 m2a(-2.0f * alpha.hi, -2.0f * alpha.lo);
#pragma unroll
    for (int n = 0; n <= L; ++n) {
        b.v[n] = pre * F[n];
        if (n < L) pre = pre * m2a;
    }
    return b;
}

// One warp-tile (32 bra primitive pairs at positions tl.y.. of x's class range in the exponent order
// pp_perm) against the ket pairs [kb, ke) (offsets in the partner's class range) in float-float
// arithmetic, in the FP64 core's normalisation: both sides contract the weights u = p^{-1/2} D_P
// with the unit-normalised Hermite integrals R' (base (-1)^n (2n-1)!! / R^{2n+1} beyond the
// asymptotic switch, df_table_base below it; the warp takes the table only when one of its lanes
// needs it), the bra field is scaled by (sqrt(pi)/2) p^{-1/2} once per tile in FP64 and the ket
// field by (sqrt(pi)/2) q^{-1/2} once per flushed batch.
template <int LP, int LQ>
__device__ __forceinline__ void jtile_df(const Dev& d, const int2 tl, const int kb, const int ke, const float tau,
                                         const int lane, const DfKetBuf& kbuf)
{
    constexpr int NP = nh(LP), NQ = nh(LQ), L = LP + LQ, NR = nh(LP + LQ);
    constexpr int kBatch = 32 / NQ;
    const int pr = tl.x >> 1;
    const int x = (tl.x & 1) ? d.pair_y[pr] : d.pair_x[pr];
    const int y = (tl.x & 1) ? d.pair_x[pr] : d.pair_y[pr];
    const int bra_end = d.frag_pp0[x * kClasses + LP] + d.frag_npp[x * kClasses + LP];
    const bool valid = tl.y + lane < bra_end;
    const int Pl = d.pp_perm[LP][valid ? tl.y + lane : tl.y];
    const int nP = d.n_pp[LP], nQ = d.n_pp[LQ];
    const int kc = d.frag_pp0[y * kClasses + LQ];
    const int k0 = kc + kb;
    const int k1 = kc + min(ke, d.frag_npp[y * kClasses + LQ]);
    if (k0 >= k1) return;  // a ket chunk beyond the partner's range
    const float4 Ph = d.pp_Phi[LP][Pl], Plo = d.pp_Plo[LP][Pl];
    const df64 Px(Ph.x, Plo.x), Py(Ph.y, Plo.y), Pz(Ph.z, Plo.z), p(Ph.w, Plo.w);
    const float2 sqp2 = d.pp_sqdf[LP][Pl];
    const df64 sqp(sqp2.x, sqp2.y);
    const float4 Pf = d.pp_Pf[LP][Pl];
    const float qP = valid ? d.pp_Q[LP][Pl] : 0.0f;
    df64 DP[NP];
    dfacc JP[NP];
    double JP64[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        DP[i] = valid ? ld_df(d.pp_udf[LP] + (size_t)i * nP + Pl) : df64(0.0f, 0.0f);
        JP[i] = dfacc{0.0f, 0.0f};
        JP64[i] = 0.0;
    }
    const float4* __restrict__ QH = d.pp_Phi[LQ];
    const float4* __restrict__ QL = d.pp_Plo[LQ];
    const float4* __restrict__ QPf = d.pp_Pf[LQ];
    const float2* __restrict__ QSQ = d.pp_sqdf[LQ];
    const float* __restrict__ QQ = d.pp_Q[LQ];
    const float2* __restrict__ QD = d.pp_udf[LQ];
    double* __restrict__ QJ = d.pp_Jh[LQ];
    int since_flush = 0;
    int cnt = 0;  // kets staged in kbuf
    for (int k = k0; k < k1; ++k) {
        const float qQ = __ldg(QQ + k);
        const bool keep = qP * qQ >= tau;
        if (!__any_sync(0xffffffffu, keep)) continue;
        const float4 Qh = __ldg(QH + k), Ql = __ldg(QL + k);
        const float4 Qf = __ldg(QPf + k);
        df64 DQ[NQ];
#pragma unroll
        for (int j = 0; j < NQ; ++j) DQ[j] = ld_df(QD + (size_t)j * nQ + k);
        const df64 X = Px - df64(Qh.x, Ql.x), Y = Py - df64(Qh.y, Ql.y), Z = Pz - df64(Qh.z, Ql.z);
        const df64 R2 = fma(X, X, fma(Y, Y, Z * Z));
        const float Xf = Pf.x - Qf.x, Yf = Pf.y - Qf.y, Zf = Pf.z - Qf.z;
        const float R2f = fmaf(Xf, Xf, fmaf(Yf, Yf, Zf * Zf));
        const float pqf = Pf.w * Qf.w, sf = Pf.w + Qf.w;
        const bool asym = pqf * R2f >= (float)kBoysTmax * sf;
        // asymptotic (point-multipole) base for every lane; lanes below the switch overwrite it
        const df64 yv = rsqrt_df_seed(R2, rsqrt_approx(R2.hi));
        df64 base[L + 1];
        base[0] = keep ? yv : df64(0.0f, 0.0f);
        if constexpr (L > 0) {
            const df64 ny2 = -(yv * yv);
            base[1] = base[0] * ny2;
#pragma unroll
            for (int n = 1; n < L; ++n) base[n + 1] = base[n] * mul_df_f(ny2, (float)(2 * n + 1));
        }
        if (!__all_sync(0xffffffffu, asym)) {
            if (!asym) {
                const float2 sqq = __ldg(QSQ + k);
                const BaseDf<L> t = df_table_base<L>(d.boysdf, p, df64(Qh.w, Ql.w), sqp, df64(sqq.x, sqq.y), R2,
                                                     __fdividef(pqf, sf) * R2f);
#pragma unroll
                for (int n = 0; n <= L; ++n) base[n] = keep ? t.v[n] : df64(0.0f, 0.0f);
            }
        }
        df64 R[NR];
        md_R<L, df64>(R, base, X, Y, Z);
        // field on the bra pair (registers, unnormalised sums)
        static_for<NP>([&](auto I) {
            constexpr TUV a = htuv(decltype(I)::value);
            static_for<NQ>([&](auto Jc) {
                constexpr TUV b = htuv(decltype(Jc)::value);
                constexpr int rr = hidx(a.t + b.t, a.u + b.u, a.v + b.v);
                if constexpr (((b.t + b.u + b.v) & 1) != 0)
                    acc_prod(JP[decltype(I)::value], -R[rr], DQ[decltype(Jc)::value]);
                else
                    acc_prod(JP[decltype(I)::value], R[rr], DQ[decltype(Jc)::value]);
            });
        });
        // field on the ket pair: this lane's float-float partial sums (unnormalised), staged for the batch
        float2* row = kbuf.v + lane * kDfBufLd + cnt * NQ;
        static_for<NQ>([&](auto Jc) {
            constexpr TUV b = htuv(decltype(Jc)::value);
            dfacc s{0.0f, 0.0f};
            static_for<NP>([&](auto I) {
                constexpr TUV a = htuv(decltype(I)::value);
                acc_prod(s, R[hidx(a.t + b.t, a.u + b.u, a.v + b.v)], DP[decltype(I)::value]);
            });
            if ((b.t + b.u + b.v) & 1) row[decltype(Jc)::value] = make_float2(-s.s, -s.c);
            else row[decltype(Jc)::value] = make_float2(s.s, s.c);
        });
        if (lane == 0) kbuf.k[cnt] = k;
        if (++cnt == kBatch) {
            df_ketbuf_flush<NQ>(kbuf, cnt, QJ, (size_t)nQ, d.pp_rp[LQ], lane);
            cnt = 0;
        }
        if (++since_flush == kFlushKets) {
            since_flush = 0;
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                JP64[i] += f2d(JP[i].s) + f2d(JP[i].c);
                JP[i] = dfacc{0.0f, 0.0f};
            }
        }
    }
    if (cnt > 0) df_ketbuf_flush<NQ>(kbuf, cnt, QJ, (size_t)nQ, d.pp_rp[LQ], lane);
    if (valid) {
        const double aP = kSqrtPiHalf * d.pp_rp[LP][Pl];
#pragma unroll
        for (int i = 0; i < NP; ++i)
            atomicAdd(d.pp_Jh[LP] + (size_t)i * nP + Pl, (JP64[i] + (f2d(JP[i].s) + f2d(JP[i].c))) * aP);
    }
}

template <int LP, int LQ>
__global__ void __launch_bounds__(128) k_jengine_df(Dev d, const int2* __restrict__ tiles, int n_tiles, float tau)
{
    __shared__ float2 kv[4 * kDfBufWarp];
    __shared__ int kk[4 * 32];
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (warp >= n_tiles) return;
    const int w = threadIdx.x >> 5;
    jtile_df<LP, LQ>(d, tiles[warp], 0, INT_MAX, tau, threadIdx.x & 31, DfKetBuf{kv + w * kDfBufWarp, kk + w * 32});
}

// Persistent float-float J-engine over the s/p classes: warps take cost-sorted items from a queue
// (item encoding in internal.hpp) until it is empty.
__global__ void __launch_bounds__(128) k_jengine_df_persistent(Dev d, const int4* __restrict__ items, int n_items,
                                                               int* __restrict__ next, float tau)
{
    __shared__ float2 kv[4 * kDfBufWarp];
    __shared__ int kk[4 * 32];
    const int lane = threadIdx.x & 31;
    const DfKetBuf kbuf{kv + (threadIdx.x >> 5) * kDfBufWarp, kk + (threadIdx.x >> 5) * 32};
    for (;;) {
        int i = 0;
        if (lane == 0) i = atomicAdd(next, 1);
        i = __shfl_sync(0xffffffffu, i, 0);
        if (i >= n_items) return;
        const int4 it = items[i];
        const int2 tl = make_int2(it.x, it.y);
        const int kb = it.z, ke = jitem_ket_end(it);
        switch (jitem_class(it)) {
            case 0 * kClasses + 0: jtile_df<0, 0>(d, tl, kb, ke, tau, lane, kbuf); break;
            case 1 * kClasses + 0: jtile_df<1, 0>(d, tl, kb, ke, tau, lane, kbuf); break;
            case 1 * kClasses + 1: jtile_df<1, 1>(d, tl, kb, ke, tau, lane, kbuf); break;
            case 2 * kClasses + 0: jtile_df<2, 0>(d, tl, kb, ke, tau, lane, kbuf); break;
            case 2 * kClasses + 1: jtile_df<2, 1>(d, tl, kb, ke, tau, lane, kbuf); break;
            case 2 * kClasses + 2: jtile_df<2, 2>(d, tl, kb, ke, tau, lane, kbuf); break;
            default: break;
        }
    }
}

template <int LP, int LQ>
void launch_df_one(const Dev& d, const int2* t, int n, float tau, cudaStream_t s)
{
    if (n <= 0) return;
    const int warps_per_block = 4;
    k_jengine_df<LP, LQ><<<(n + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, s>>>(d, t, n, tau);
    note_launches(1);
}

// df64 copies of the FP64 pair data and Boys table (once per geometry)
__global__ void k_split_pairs(const double4_32a* __restrict__ P, float4* hi, float4* lo, int n)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const double4_32a v = P[g];
    const float hx = (float)v.x, hy = (float)v.y, hz = (float)v.z, hw = (float)v.w;
    hi[g] = make_float4(hx, hy, hz, hw);
    lo[g] = make_float4((float)(v.x - hx), (float)(v.y - hy), (float)(v.z - hz), (float)(v.w - hw));
}

__global__ void k_split_sqrt_p(const double4_32a* __restrict__ P, const double* __restrict__ rp, float2* out, int n)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const double v = P[g].w * rp[g];  // sqrt(p) = p p^{-1/2}
    const float h = (float)v;
    out[g] = make_float2(h, (float)(v - h));
}

__global__ void k_split_array(const double* __restrict__ a, float2* out, size_t n)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double v = a[i];
        const float h = (float)v;
        out[i] = make_float2(h, (float)(v - h));
    }
}

}  // namespace

cudaError_t launch_df_setup(const Dev& d, float4* const Phi[kClasses], float4* const Plo[kClasses],
                            float2* const sqdf[kClasses], float2* boysdf, cudaStream_t s)
{
    for (int L = 0; L < kClasses; ++L) {
        if (d.n_pp[L] == 0) continue;
        k_split_pairs<<<(d.n_pp[L] + 127) / 128, 128, 0, s>>>(d.pp_P[L], Phi[L], Plo[L], d.n_pp[L]);
        k_split_sqrt_p<<<(d.n_pp[L] + 127) / 128, 128, 0, s>>>(d.pp_P[L], d.pp_rp[L], sqdf[L], d.n_pp[L]);
        note_launches(2);
    }
    const size_t nb = (size_t)kBoysRows * kBoysRowLen;
    k_split_array<<<(unsigned)((nb + 255) / 256), 256, 0, s>>>(d.boys, boysdf, nb);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_df_density(const Dev& d, cudaStream_t s)
{
    for (int L = 0; L < kClasses; ++L) {
        const size_t n = (size_t)nh(L) * d.n_pp[L];
        if (n == 0) continue;
        k_split_array<<<(unsigned)std::min<size_t>((n + 255) / 256, 2048), 256, 0, s>>>(d.pp_u[L], d.pp_udf[L], n);
        note_launches(1);
    }
    return cudaGetLastError();
}

cudaError_t jengine_df_persistent_grid(int* blocks_per_sm)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_jengine_df_persistent, 128, 0);
}

cudaError_t launch_jengine_df_persistent(const Dev& d, const JQueue& q, float tau, cudaStream_t s)
{
    if (q.n <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(q.next, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    const int blocks = std::max(1, std::min(q.grid, (q.n + 3) / 4));
    k_jengine_df_persistent<<<blocks, 128, 0, s>>>(d, q.items, q.n, q.next, tau);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_jengine_df_class(const Dev& d, int LP, int LQ, const int2* t, int n, float tau, cudaStream_t s)
{
    switch (LP * kClasses + LQ) {
        case 0 * kClasses + 0: launch_df_one<0, 0>(d, t, n, tau, s); break;
        case 1 * kClasses + 0: launch_df_one<1, 0>(d, t, n, tau, s); break;
        case 1 * kClasses + 1: launch_df_one<1, 1>(d, t, n, tau, s); break;
        case 2 * kClasses + 0: launch_df_one<2, 0>(d, t, n, tau, s); break;
        case 2 * kClasses + 1: launch_df_one<2, 1>(d, t, n, tau, s); break;
        case 2 * kClasses + 2: launch_df_one<2, 2>(d, t, n, tau, s); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Class pairs with L_P <= 2 in df64; the others (d shells) in native FP64.
cudaError_t launch_jengine_df(const Dev& d, const int2* tiles[kClasses][kClasses], const int* n_tiles, float tau,
                              cudaStream_t s)
{
#define FEF_JD(LP, LQ) launch_df_one<LP, LQ>(d, tiles[LP][LQ], n_tiles[LP * kClasses + LQ], tau, s)
    FEF_JD(0, 0); FEF_JD(1, 0); FEF_JD(1, 1); FEF_JD(2, 0); FEF_JD(2, 1); FEF_JD(2, 2);
#undef FEF_JD
    return cudaGetLastError();
}

}  // namespace fef
