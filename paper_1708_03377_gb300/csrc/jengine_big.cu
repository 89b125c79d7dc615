// J-engine classes with L = L_P + L_Q >= 5 (shell pairs with d functions; up to (dd|dd), L = 8).
// Same contraction as the register kernels of jengine.cu (McMurchie-Davidson Hermite field of the
// partner fragment's density, paper Eq. dp2e / Eq. wc), but each lane keeps its nh(L) Hermite
// integrals R_{tuv} in a lane-strided slice of shared memory (too many for registers at L >= 5), the
// warp-uniform ket Hermite density is staged in shared memory, and the field on the ket pair is
// reduced across the warp in chunks of 5 components.  Two warps per block.
#include <algorithm>
#include <climits>
#include <type_traits>

#include "common.cuh"
#include "internal.hpp"

namespace fef {

namespace {

constexpr int kBigWarps = 2;

template <int LP, int LQ>
__host__ __device__ constexpr int big_slice()  // Reals per warp: R slices of 32 lanes + ket density (+ pad to 2)
{
    return 32 * nh(LP + LQ) + ((nh(LQ) + 1) & ~1);
}

// The ket-side field of the FP32 core is scaled by the ket's k = k_hi + k_lo (kQ, a float pair) as it
// leaves FP32; the FP64 core passes (1, 0).
template <int NP, int NQ, typename Real, typename RArr>
__device__ __forceinline__ void contract_big(RArr R, const Real* DP, const Real* DQ, Real* JP,
                                             double* __restrict__ QJ, size_t nQ, int k, int lane, float2 kQ)
{
    static_for<NP>([&](auto I) {
        constexpr TUV a = htuv(decltype(I)::value);
        Real acc = JP[decltype(I)::value];
        static_for<NQ>([&](auto Jc) {
            constexpr TUV b = htuv(decltype(Jc)::value);
            constexpr int r = hidx(a.t + b.t, a.u + b.u, a.v + b.v);
            if constexpr (((b.t + b.u + b.v) & 1) != 0)
                acc = fma(-R[r], DQ[decltype(Jc)::value], acc);
            else
                acc = fma(R[r], DQ[decltype(Jc)::value], acc);
        });
        JP[decltype(I)::value] = acc;
    });
    constexpr int CH = 5;
    static_for<(NQ + CH - 1) / CH>([&](auto C) {
        constexpr int j0 = decltype(C)::value * CH;
        Real sq[CH];
        static_for<CH>([&](auto Jj) {
            constexpr int j = j0 + decltype(Jj)::value;
            if constexpr (j < NQ) {
                constexpr TUV b = htuv(j);
                Real s = Real(0);
                static_for<NP>([&](auto I) {
                    constexpr TUV a = htuv(decltype(I)::value);
                    s = fma(R[hidx(a.t + b.t, a.u + b.u, a.v + b.v)], DP[decltype(I)::value], s);
                });
                sq[decltype(Jj)::value] = ((b.t + b.u + b.v) & 1) ? -s : s;
            } else {
                sq[decltype(Jj)::value] = Real(0);
            }
        });
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            static_for<CH>([&](auto Jj) {
                sq[decltype(Jj)::value] += __shfl_xor_sync(0xffffffffu, sq[decltype(Jj)::value], o);
            });
        if (lane == 0)
            static_for<CH>([&](auto Jj) {
                constexpr int j = j0 + decltype(Jj)::value;
                if constexpr (j < NQ) {
                    if constexpr (std::is_same<Real, float>::value)
                        atomicAdd(QJ + (size_t)j * nQ + k,
                                  f2d(fmaf(sq[decltype(Jj)::value], kQ.y, sq[decltype(Jj)::value] * kQ.x)));
                    else
                        atomicAdd(QJ + (size_t)j * nQ + k, f2d(sq[decltype(Jj)::value]));
                }
            });
    });
}

// Real = double: full FP64 build on pp_Dh.  Real = float: the FP32 core on the FP32 records (the same
// as the register classes of jengine.cu: weights u = p^{-1/2} (D_P - D_P^ref) with charge-conserving
// rounding, the unit-normalised Hermite integrals R' with the point-multipole form beyond the Boys
// switch, each bra centre relative to the ket fragment's first atom, the scale factors
// k = (sqrt(pi)/2) p^{-1/2} applied as float pairs), the bra field flushed to FP64 every 16 ket pairs.
// One warp-tile (32 bra primitive pairs from tl.y) against the ket pairs [kb, ke) (offsets in the
// partner's class range); sm = this warp's shared-memory slice of big_slice<LP, LQ>() Reals.
template <int LP, int LQ, typename Real>
__device__ __forceinline__ void jtile_big(const Dev& d, const int2 tl, const int kb, const int ke, const float tau,
                                          const int lane, Real* sm)
{
    constexpr bool F32 = std::is_same<Real, float>::value;
    constexpr int NP = nh(LP), NQ = nh(LQ), L = LP + LQ;
    constexpr int RP = rec32_len(LP), RQ = rec32_len(LQ);
    LaneSlice<Real> R{sm + lane};
    Real* DQ = sm + 32 * nh(L);
    const int pr = tl.x >> 1;
    const int x = (tl.x & 1) ? d.pair_y[pr] : d.pair_x[pr];
    const int y = (tl.x & 1) ? d.pair_x[pr] : d.pair_y[pr];
    const int bra_end = d.frag_pp0[x * kClasses + LP] + d.frag_npp[x * kClasses + LP];
    const int Pg = tl.y + lane;
    const bool valid = Pg < bra_end;
    const int Pl = valid ? Pg : tl.y;
    const int nP = d.n_pp[LP], nQ = d.n_pp[LQ];
    const float qP = valid ? d.pp_Q[LP][Pl] : 0.0f;
    Real DP[NP], JP[NP];
    double JP64[NP];
    const double4_32a Pd = d.pp_P[LP][Pl];
    float4 Pf{};
    float px = 0.f, py = 0.f, pz = 0.f, pP = 0.f;
    double kP = 0.0;  // bra field scale k_hi + k_lo (FP32 core)
    if constexpr (F32) {
        const float* __restrict__ brec = d.pp_rec32[LP] + (size_t)Pl * RP;
        const double* ay = d.atom_xyz + 3 * d.frag_atom0[y];
        px = (float)(Pd.x - ay[0]);
        py = (float)(Pd.y - ay[1]);
        pz = (float)(Pd.z - ay[2]);
        pP = (float)Pd.w;
        kP = f2d(brec[4]) + f2d(brec[5]);
#pragma unroll
        for (int i = 0; i < NP; ++i) DP[i] = valid ? brec[8 + i] : 0.0f;
    } else {
        Pf = d.pp_Pf[LP][Pl];
#pragma unroll
        for (int i = 0; i < NP; ++i) DP[i] = valid ? d.pp_Dh[LP][(size_t)i * nP + Pl] : 0.0;
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        JP[i] = Real(0);
        JP64[i] = 0.0;
    }
    const int kc = d.frag_pp0[y * kClasses + LQ];
    const int k0 = kc + kb;
    const int k1 = kc + min(ke, d.frag_npp[y * kClasses + LQ]);
    double* __restrict__ QJ = d.pp_Jh[LQ];
    const float* __restrict__ QR = d.pp_rec32[LQ];
    int since_flush = 0;
    for (int k = k0; k < k1; ++k) {
        const float qQ = __ldg(d.pp_Q[LQ] + k);
        const bool keep = qP * qQ >= tau;
        if (!__any_sync(0xffffffffu, keep)) continue;
        __syncwarp();
        for (int j = lane; j < NQ; j += 32) {
            if constexpr (F32)
                DQ[j] = __ldg(QR + (size_t)k * RQ + 8 + j);
            else
                DQ[j] = __ldg(d.pp_Dh[LQ] + (size_t)j * nQ + k);
        }
        __syncwarp();
        Real base[L + 1];
        Real X, Y, Z;
        float2 kQ = make_float2(1.0f, 0.0f);
        if constexpr (F32) {
            const float4 q0 = __ldg(reinterpret_cast<const float4*>(QR + (size_t)k * RQ));
            kQ = __ldg(reinterpret_cast<const float2*>(QR + (size_t)k * RQ + 4));
            X = px - q0.x;
            Y = py - q0.y;
            Z = pz - q0.z;
            const float R2 = fmaf(X, X, fmaf(Y, Y, Z * Z));
            const float pq = pP * q0.w, sq = pP + q0.w;
            // point multipoles beyond the switch (R'^{(n)} = (-1)^n (2n-1)!! / R^{2n+1}); table below it
            const float yv = keep ? rsqrt_nr(R2) : 0.0f;
            const float ny2 = -(yv * yv);
            base[0] = yv;
#pragma unroll
            for (int n = 0; n < L; ++n) base[n + 1] = base[n] * (float(2 * n + 1) * ny2);
            const bool asym = pq * R2 >= kFp32SwitchHigh * sq;
            if (!__all_sync(0xffffffffu, asym)) {
                if (!asym) {
                    const Base32<L> t = fp32_table_base<L>(d.boys32, pq, sq, R2);
#pragma unroll
                    for (int n = 0; n <= L; ++n) base[n] = keep ? t.v[n] : 0.0f;
                }
            }
        } else {
            const double4_32a Qd = d.pp_P[LQ][k];
            const float4 Qf = __ldg(d.pp_Pf[LQ] + k);
            X = Pd.x - Qd.x;
            Y = Pd.y - Qd.y;
            Z = Pd.z - Qd.z;
            const double r = rsqrt(Pd.w + Qd.w);
            const double alpha = Pd.w * Qd.w * (r * r);
            const float Xf = Pf.x - Qf.x, Yf = Pf.y - Qf.y, Zf = Pf.z - Qf.z;
            const float Tf = __fdividef(Pf.w * Qf.w, Pf.w + Qf.w) * fmaf(Xf, Xf, fmaf(Yf, Yf, Zf * Zf));
            double F[L + 1];
            boys_fp64<L>(d.boys, alpha * fma(X, X, fma(Y, Y, Z * Z)), boys_row(Tf), F);
            double pre = keep ? r : 0.0;
#pragma unroll
            for (int n = 0; n <= L; ++n) {
                base[n] = pre * F[n];
                pre *= -2.0 * alpha;
            }
        }
        md_R<L, Real>(R, base, X, Y, Z);
        contract_big<NP, NQ, Real>(R, DP, DQ, JP, QJ, (size_t)nQ, k, lane, kQ);
        if constexpr (F32) {
            if (++since_flush == 16) {
                since_flush = 0;
#pragma unroll
                for (int i = 0; i < NP; ++i) {
                    JP64[i] += f2d(JP[i]);
                    JP[i] = 0.0f;
                }
            }
        }
    }
    if (valid) {
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            const double j = JP64[i] + f2d(JP[i]);
            atomicAdd(d.pp_Jh[LP] + (size_t)i * nP + Pg, F32 ? j * kP : j);
        }
    }
}

template <int LP, int LQ, typename Real>
__global__ void __launch_bounds__(32 * kBigWarps) k_jengine_big(Dev d, const int2* __restrict__ tiles, int n_tiles,
                                                                 float tau)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int wib = threadIdx.x >> 5;
    const int warp = blockIdx.x * kBigWarps + wib;
    if (warp >= n_tiles) return;
    Real* sm = reinterpret_cast<Real*>(smraw) + wib * big_slice<LP, LQ>();
    jtile_big<LP, LQ, Real>(d, tiles[warp], 0, INT_MAX, tau, threadIdx.x & 31, sm);
}

// Persistent kernel over the classes with L_P + L_Q >= 5: warps take cost-sorted items from a queue
// (item encoding in internal.hpp); every warp owns a slice of `slice` Reals, the largest class's.
template <typename Real>
__global__ void __launch_bounds__(32 * kBigWarps) k_jengine_big_persistent(Dev d, const int4* __restrict__ items,
                                                                            int n_items, int* __restrict__ next,
                                                                            float tau, int slice)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int lane = threadIdx.x & 31;
    Real* sm = reinterpret_cast<Real*>(smraw) + (threadIdx.x >> 5) * slice;
    for (;;) {
        int i = 0;
        if (lane == 0) i = atomicAdd(next, 1);
        i = __shfl_sync(0xffffffffu, i, 0);
        if (i >= n_items) return;
        const int4 it = items[i];
        const int2 tl = make_int2(it.x, it.y);
        const int kb = it.z, ke = jitem_ket_end(it);
        switch (jitem_class(it)) {
            case 3 * kClasses + 2: jtile_big<3, 2, Real>(d, tl, kb, ke, tau, lane, sm); break;
            case 3 * kClasses + 3: jtile_big<3, 3, Real>(d, tl, kb, ke, tau, lane, sm); break;
            case 4 * kClasses + 1: jtile_big<4, 1, Real>(d, tl, kb, ke, tau, lane, sm); break;
            case 4 * kClasses + 2: jtile_big<4, 2, Real>(d, tl, kb, ke, tau, lane, sm); break;
            case 4 * kClasses + 3: jtile_big<4, 3, Real>(d, tl, kb, ke, tau, lane, sm); break;
            case 4 * kClasses + 4: jtile_big<4, 4, Real>(d, tl, kb, ke, tau, lane, sm); break;
            default: break;
        }
        __syncwarp();
    }
}

template <int LP, int LQ>
void launch_big(const Dev& d, const int2* t, int n, float tau, int fp32, cudaStream_t s)
{
    if (n <= 0) return;
    const int blocks = (n + kBigWarps - 1) / kBigWarps;
    if (fp32) {
        const size_t smem = (size_t)kBigWarps * big_slice<LP, LQ>() * sizeof(float);
        cudaFuncSetAttribute(k_jengine_big<LP, LQ, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_jengine_big<LP, LQ, float><<<blocks, 32 * kBigWarps, smem, s>>>(d, t, n, tau);
    } else {
        const size_t smem = (size_t)kBigWarps * big_slice<LP, LQ>() * sizeof(double);
        cudaFuncSetAttribute(k_jengine_big<LP, LQ, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_jengine_big<LP, LQ, double><<<blocks, 32 * kBigWarps, smem, s>>>(d, t, n, tau);
    }
    note_launches(1);
}

}  // namespace

int jengine_big_slice(int LP, int LQ) { return 32 * nh(LP + LQ) + ((nh(LQ) + 1) & ~1); }

// The dynamic shared-memory limit of the persistent kernel is raised once to the largest class's
// need, so that queues of any context (smaller slices) can be launched.
cudaError_t jengine_big_persistent_grid(int fp32, int smem_slice, int* blocks_per_sm)
{
    const size_t real = fp32 ? sizeof(float) : sizeof(double);
    const size_t smem = (size_t)kBigWarps * smem_slice * real;
    const size_t smem_max = (size_t)kBigWarps * big_slice<kClasses - 1, kClasses - 1>() * real;
    if (smem > smem_max) return cudaErrorInvalidValue;
    const void* k = fp32 ? (const void*)k_jengine_big_persistent<float> : (const void*)k_jengine_big_persistent<double>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, 32 * kBigWarps, smem);
}

cudaError_t launch_jengine_big_persistent(const Dev& d, int fp32, const JQueue& q, float tau, cudaStream_t s)
{
    if (q.n <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(q.next, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    const int blocks = std::max(1, std::min(q.grid, (q.n + kBigWarps - 1) / kBigWarps));
    const size_t smem = (size_t)kBigWarps * q.smem_slice * (fp32 ? sizeof(float) : sizeof(double));
    if (fp32)
        k_jengine_big_persistent<float><<<blocks, 32 * kBigWarps, smem, s>>>(d, q.items, q.n, q.next, tau, q.smem_slice);
    else
        k_jengine_big_persistent<double><<<blocks, 32 * kBigWarps, smem, s>>>(d, q.items, q.n, q.next, tau, q.smem_slice);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_jengine_big_class(const Dev& d, int LP, int LQ, const int2* t, int n, float tau, int fp32,
                                     cudaStream_t s)
{
    switch (LP * kClasses + LQ) {
        case 3 * kClasses + 2: launch_big<3, 2>(d, t, n, tau, fp32, s); break;
        case 3 * kClasses + 3: launch_big<3, 3>(d, t, n, tau, fp32, s); break;
        case 4 * kClasses + 1: launch_big<4, 1>(d, t, n, tau, fp32, s); break;
        case 4 * kClasses + 2: launch_big<4, 2>(d, t, n, tau, fp32, s); break;
        case 4 * kClasses + 3: launch_big<4, 3>(d, t, n, tau, fp32, s); break;
        case 4 * kClasses + 4: launch_big<4, 4>(d, t, n, tau, fp32, s); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_jengine_big(const Dev& d, const int2* tiles[kClasses][kClasses], const int* n_tiles, float tau,
                               int fp32, cudaStream_t s)
{
#define FEF_JB(LP, LQ) launch_big<LP, LQ>(d, tiles[LP][LQ], n_tiles[LP * kClasses + LQ], tau, fp32, s)
    FEF_JB(3, 2); FEF_JB(3, 3); FEF_JB(4, 1); FEF_JB(4, 2); FEF_JB(4, 3); FEF_JB(4, 4);
#undef FEF_JB
    return cudaGetLastError();
}

}  // namespace fef
