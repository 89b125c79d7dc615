// The inter-fragment Coulomb field of the FEF Fock build (paper, "Fragment Mean Field",
// Eq. wc: omega_x = h~ + 2 v, with v of Eq. dp2e; 2 v = J[D^y] for the closed-shell density
// D^y = 2 C_occ C_occ^T).
//
// J-engine (McMurchie-Davidson Hermite contraction; Ahmadi & Almlof 1995, White & Head-Gordon 1996):
//   Hermite density of every primitive pair Q (shells c <= d of fragment y, weight 2 for c != d):
//       D_Q[t'u'v'] = sum_{lambda in c, sigma in d} w D^y_{lambda sigma} E^{lambda sigma}_{t'u'v'}(Q)
//   Hermite Coulomb field of a bra pair P of fragment x:
//       J_P[tuv] = sum_Q 2 pi^{5/2}/(p q sqrt(p+q)) sum_{t'u'v'} (-1)^{t'+u'+v'} R_{t+t',u+u',v+v'} D_Q[t'u'v']
//   and, from the same R, the field of x on Q:  J_Q[t'u'v'] += (-1)^{t'+u'+v'} sum_{tuv} R_{...} D_P[tuv].
//   J^x_{mu nu} = sum_{P in (a,b)} sum_tuv E^{mu nu}_{tuv}(P) J_P[tuv].
// The ERIs (mu nu|lambda sigma) are never formed.  Densities and fields are pre/post-scaled by
// c/p with c = sqrt(2 pi^{5/2}) so that each primitive quartet only needs rsqrt(p+q).
#include <algorithm>
#include <climits>

#include "common.cuh"
#include "internal.hpp"

namespace fef {

// ------------------------------------------------------------------------------------------ densities
// Hermite density of one primitive pair g of class L (shell pair of angular momenta LA, LB known at
// compile time, so that the expansion coefficients stay in registers):
//   Dh_P[tuv] = (2 pi^{5/2} K / p) sum_{mu in a, nu in b} w D_{mu nu} E^{mu nu}_tuv(P),
// w = 2 for a != b (both triangles), and the J-engine weights u = p^{-1/2} Dh_P.
template <int LA, int LB>
__device__ __forceinline__ void hermite_density_pair(const Dev& d, int L, int g, const double* __restrict__ D)
{
    constexpr int NH = nh(LA + LB);
    const int npp = d.n_pp[L];
    const int sp = d.pp_sp[L][g];
    const int sa = d.sp_a[sp], sb = d.sp_b[sp];
    const int x = frag_of_shellpair(d, sp);
    const double* A = d.atom_xyz + 3 * d.sh_atom[sa];
    const double* B = d.atom_xyz + 3 * d.sh_atom[sb];
    const double4_32a P = d.pp_P[L][g];
    const double p = P.w;
    double E[3][3][3][5];
    md_E1(LA, LB, p, P.x - A[0], P.x - B[0], E[0]);
    md_E1(LA, LB, p, P.y - A[1], P.y - B[1], E[1]);
    md_E1(LA, LB, p, P.z - A[2], P.z - B[2], E[2]);
    const int n = d.frag_nao[x];
    const double* Dx = D + d.frag_moff[x];
    const int ao0 = d.frag_ao0[x];
    const double w = (sa == sb) ? 1.0 : 2.0;
    const int mu0 = d.sh_ao[sa], nu0 = d.sh_ao[sb];
    double acc[NH];
#pragma unroll
    for (int k = 0; k < NH; ++k) acc[k] = 0.0;
#pragma unroll
    for (int ia = 0; ia < ncart(LA); ++ia) {
        int ax, ay, az;
        cart_of(LA, ia, ax, ay, az);
        const int mu = mu0 + ia;
#pragma unroll
        for (int ib = 0; ib < ncart(LB); ++ib) {
            int bx, by, bz;
            cart_of(LB, ib, bx, by, bz);
            const int nu = nu0 + ib;
            const double dmn = w * Dx[mu * n + nu] * d.ao_scale[ao0 + mu] * d.ao_scale[ao0 + nu];
#pragma unroll
            for (int t = 0; t <= LA + LB; ++t)
#pragma unroll
                for (int u = 0; u <= LA + LB - t; ++u)
#pragma unroll
                    for (int v = 0; v <= LA + LB - t - u; ++v)
                        if (t <= ax + bx && u <= ay + by && v <= az + bz)
                            acc[hidx(t, u, v)] += dmn * E[0][ax][bx][t] * E[1][ay][by][u] * E[2][az][bz][v];
        }
    }
    const double sc = d.pp_K[L][g] * kSqrt2Pi52 / p;
    const double rp = d.pp_rp[L][g];
#pragma unroll
    for (int k = 0; k < NH; ++k) {
        d.pp_Dh[L][(size_t)k * npp + g] = acc[k] * sc;
        d.pp_u[L][(size_t)k * npp + g] = acc[k] * sc * rp;
    }
}

// Systems of s and p shells only (the smaller register footprint), and the general kernel.
__global__ void k_hermite_density_sp(Dev d, int L, const double* __restrict__ D)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= d.n_pp[L]) return;
    const int sp = d.pp_sp[L][g];
    switch (d.sh_l[d.sp_a[sp]] * 3 + d.sh_l[d.sp_b[sp]]) {
        case 0: hermite_density_pair<0, 0>(d, L, g, D); break;
        case 1: hermite_density_pair<0, 1>(d, L, g, D); break;
        case 3: hermite_density_pair<1, 0>(d, L, g, D); break;
        default: hermite_density_pair<1, 1>(d, L, g, D); break;
    }
}

__global__ void k_hermite_density(Dev d, int L, const double* __restrict__ D)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= d.n_pp[L]) return;
    const int sp = d.pp_sp[L][g];
    switch (d.sh_l[d.sp_a[sp]] * 3 + d.sh_l[d.sp_b[sp]]) {
        case 0: hermite_density_pair<0, 0>(d, L, g, D); break;
        case 1: hermite_density_pair<0, 1>(d, L, g, D); break;
        case 2: hermite_density_pair<0, 2>(d, L, g, D); break;
        case 3: hermite_density_pair<1, 0>(d, L, g, D); break;
        case 4: hermite_density_pair<1, 1>(d, L, g, D); break;
        case 5: hermite_density_pair<1, 2>(d, L, g, D); break;
        case 6: hermite_density_pair<2, 0>(d, L, g, D); break;
        case 7: hermite_density_pair<2, 1>(d, L, g, D); break;
        default: hermite_density_pair<2, 2>(d, L, g, D); break;
    }
}

cudaError_t launch_hermite_density(const Dev& d, const double* D, cudaStream_t s)
{
    for (int L = 0; L < kClasses; ++L)
        if (d.n_pp[L] > 0) {
            if (d.max_l <= 1)
                k_hermite_density_sp<<<(d.n_pp[L] + 127) / 128, 128, 0, s>>>(d, L, D);
            else
                k_hermite_density<<<(d.n_pp[L] + 127) / 128, 128, 0, s>>>(d, L, D);
            note_launches(1);
        }
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------ J-engine
// Both contractions of one primitive quartet with compile-time Hermite indices:
//   JP[i] += sum_j (-1)^{|j|} R[i + j] DQ[j]                      (field on the bra pair, registers)
//   QJ[j][k] += (-1)^{|j|} sum_lanes sum_i R[i + j] DP[i]          (field on the ket pair)
// The ket-side field is staged per warp instead of butterfly-reduced per ket.  Lane l
// writes its partial sums of up to 32 ket components (slot = ket of the batch * NQ + component)
// into row l of a 32 x 33 shared-memory block; once the batch is full, the lane owning a slot sums
// its column over the 32 rows and adds it to global memory: 31 DADD per 32 components instead of 5
// shuffle-DADD steps for each.
constexpr int kKetBufLd = 33;
constexpr int kKetBufWarp = 32 * kKetBufLd;
struct KetBuf {
    double* v;  // [32 lanes][kKetBufLd] partial sums
    int* k;     // [32] ket pair of each batch position
};
struct KetBuf32 {  // the same for the FP32 core
    float* v;
    int* k;
};

// JP[i] += sum_j (-1)^{|j|} R[i + j] DQ[j]  (field on the lane's bra pair)
template <int NP, int NQ, typename Real>
__device__ __forceinline__ void hermite_bra(const Real* R, const Real* DQ, Real* JP)
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
}

// this lane's partial field on the ket pair, (-1)^{|j|} sum_i R[i + j] DP[i], into batch slot cnt
template <int NP, int NQ>
__device__ __forceinline__ void hermite_ket_stage(const double* R, const double* DP, const KetBuf& kb, int cnt,
                                                  int lane)
{
    double* row = kb.v + lane * kKetBufLd + cnt * NQ;
    static_for<NQ>([&](auto Jc) {
        constexpr TUV b = htuv(decltype(Jc)::value);
        double sum = 0.0;
        static_for<NP>([&](auto I) {
            constexpr TUV a = htuv(decltype(I)::value);
            sum = fma(R[hidx(a.t + b.t, a.u + b.u, a.v + b.v)], DP[decltype(I)::value], sum);
        });
        row[decltype(Jc)::value] = ((b.t + b.u + b.v) & 1) ? -sum : sum;
    });
}

template <int NP, int NQ>
__device__ __forceinline__ void hermite_ket_stage32(const float* R, const float* DP, const KetBuf32& kb, int cnt,
                                                    int lane)
{
    float* row = kb.v + lane * kKetBufLd + cnt * NQ;
    static_for<NQ>([&](auto Jc) {
        constexpr TUV b = htuv(decltype(Jc)::value);
        float sum = 0.0f;
        static_for<NP>([&](auto I) {
            constexpr TUV a = htuv(decltype(I)::value);
            sum = fmaf(R[hidx(a.t + b.t, a.u + b.u, a.v + b.v)], DP[decltype(I)::value], sum);
        });
        row[decltype(Jc)::value] = ((b.t + b.u + b.v) & 1) ? -sum : sum;
    });
}

template <int NQ>
__device__ __forceinline__ void ketbuf_flush32(const KetBuf32& kb, int cnt, double* __restrict__ QJ, size_t nQ,
                                               int lane)
{
    __syncwarp();
    if (lane < cnt * NQ) {
        float sum = 0.0f;
#pragma unroll 8
        for (int r = 0; r < 32; ++r) sum += kb.v[r * kKetBufLd + lane];
        atomicAdd(QJ + (size_t)(lane % NQ) * nQ + kb.k[lane / NQ], f2d(sum));
    }
    __syncwarp();
}

// FP64 ket flush with the ket's field scale (sqrt(pi)/2) q^{-1/2} applied to the summed column
template <int NQ>
__device__ __forceinline__ void ketbuf_flush_scaled(const KetBuf& kb, int cnt, double* __restrict__ QJ, size_t nQ,
                                                   const double* __restrict__ rq, int lane)
{
    __syncwarp();
    if (lane < cnt * NQ) {
        double sum = 0.0;
#pragma unroll 8
        for (int r = 0; r < 32; ++r) sum += kb.v[r * kKetBufLd + lane];
        const int k = kb.k[lane / NQ];
        atomicAdd(QJ + (size_t)(lane % NQ) * nQ + k, sum * (kSqrtPiHalf * __ldg(rq + k)));
    }
    __syncwarp();
}

// One warp per tile = (fragment pair, up to 32 bra primitive pairs of class LP in one member x)
// against the ket primitive pairs [kb, ke) (offsets in the class-LQ range of the other member y,
// LQ <= LP; the pair's two J directions are both produced, so the member with the larger class is
// put on the bra side).  Lane i owns the bra pair at position tl.y + i of x's class range in the
// order pp_perm (increasing exponent): its centre, Hermite density and Hermite field accumulator stay
// in registers.  Ket data are warp-uniform loads.  The field on the ket pair is staged in the warp's
// KetBuf and summed over the lanes once per batch of 32 / NQ kets.  Shell quartets with
// Q_ab Q_cd < tau contribute nothing (Schwarz screening at shell level).
//
// Boys function: for T = alpha |PQ|^2 >= kBoysTmax the asymptotic form F_n = (2n-1)!! / (2T)^n
// sqrt(pi/T) / 2 holds to the FP64 resolution of the table's own switch, and the quartet prefactor
// collapses, rsqrt(p+q) F_n(T) (-2 alpha)^n = (sqrt(pi)/2) p^{-1/2} q^{-1/2} (-1)^n (2n-1)!! / R^{2n+1}:
// the Hermite integrals of two point multipoles, one reciprocal square root per quartet.  The warp
// takes this path when all its lanes are beyond the switch (the large majority of inter-fragment
// quartets); otherwise the lanes below it evaluate the tabulated Boys function.  The per-pair factors
// are kept out of the quartet loop: both sides contract the weights u = p^{-1/2} D_P (pp_u) with the
// unit-normalised Hermite integrals R' = R / ((sqrt(pi)/2) p^{-1/2} q^{-1/2}) (base R'^{(n)} =
// (-1)^n (2n-1)!! / R^{2n+1} beyond the switch, (2/sqrt(pi)) sqrt(alpha) F_n (-2 alpha)^n below it),
// and the bra field is scaled by (sqrt(pi)/2) p^{-1/2} once per tile, the ket field by
// (sqrt(pi)/2) q^{-1/2} once per flushed batch.
// Below the asymptotic switch, the unit-normalised Hermite base of the FP64 core:
// r F_n(T) (-2 alpha)^n / (aP rq) with r = (p+q)^{-1/2}, 1/aP = inv_aP and 1/rq = q rq (see jtile_fp64).
// Kept out of line so that the asymptotic path of the quartet loop carries none of its instructions.
template <int L>
struct Base64 {
    double v[L + 1];
};
template <int L>
__device__ __noinline__ Base64<L> fp64_table_base(const double* __restrict__ boys, double p, double q, double rq,
                                                 double inv_aP, double R2, float Tf)
{
    Base64<L> b;
    const double r = rsqrt(p + q);
    const double alpha = p * q * (r * r);
    double F[L + 1];
    boys_fp64<L>(boys, alpha * R2, boys_row(Tf), F);
    double pre = r * inv_aP * (q * rq);
    const double m2a = -2.0 * alpha;
#pragma unroll
    for (int n = 0; n <= L; ++n) {
        b.v[n] = pre * F[n];
        pre *= m2a;
    }
    return b;
}

template <int LP, int LQ>
__device__ __forceinline__ void jtile_fp64(const Dev& d, const int2 tl, const int kb, const int ke, const float tau,
                                           const int lane, const KetBuf& kbuf)
{
    constexpr int kBatch = 32 / nh(LQ);
    constexpr int NP = nh(LP), NQ = nh(LQ), L = LP + LQ, NR = nh(LP + LQ);
    // tile.x = 2 * pair + swap: the bra fragment is the pair member holding the larger class
    const int pr = tl.x >> 1;
    const int x = (tl.x & 1) ? d.pair_y[pr] : d.pair_x[pr];
    const int y = (tl.x & 1) ? d.pair_x[pr] : d.pair_y[pr];
    const int bra_end = d.frag_pp0[x * kClasses + LP] + d.frag_npp[x * kClasses + LP];
    const bool valid = tl.y + lane < bra_end;
    const int Pl = d.pp_perm[LP][valid ? tl.y + lane : tl.y];
    const int nP = d.n_pp[LP], nQ = d.n_pp[LQ];
    const double4_32a Pd = d.pp_P[LP][Pl];
    const float4 Pf = d.pp_Pf[LP][Pl];
    const double rpP = d.pp_rp[LP][Pl];
    const double aP = kSqrtPiHalf * rpP;                        // bra field scale
    const double inv_aP = (1.0 / kSqrtPiHalf) * (Pd.w * rpP);   // 1/aP = (2/sqrt(pi)) sqrt(p)
    const float qP = valid ? d.pp_Q[LP][Pl] : 0.0f;
    double DP[NP], JP[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        DP[i] = valid ? d.pp_u[LP][(size_t)i * nP + Pl] : 0.0;
        JP[i] = 0.0;
    }
    const int kc = d.frag_pp0[y * kClasses + LQ];
    const int k0 = kc + kb;
    const int k1 = kc + min(ke, d.frag_npp[y * kClasses + LQ]);
    if (k0 >= k1) return;  // a ket chunk beyond the partner's range
    const double4_32a* __restrict__ QP = d.pp_P[LQ];
    const float4* __restrict__ QPf = d.pp_Pf[LQ];
    const double* __restrict__ QRP = d.pp_rp[LQ];
    const float* __restrict__ QQ = d.pp_Q[LQ];
    const double* __restrict__ QD = d.pp_u[LQ];
    double* __restrict__ QJ = d.pp_Jh[LQ];
    int cnt = 0;  // kets staged in kbuf
    for (int k = k0; k < k1; ++k) {
        const float qQ = __ldg(QQ + k);
        const bool keep = qP * qQ >= tau;
        if (!__any_sync(0xffffffffu, keep)) continue;
        const double4_32a Qd = QP[k];
        const float4 Qf = __ldg(QPf + k);
        double DQ[NQ];
#pragma unroll
        for (int j = 0; j < NQ; ++j) DQ[j] = __ldg(QD + (size_t)j * nQ + k);
        const double X = Pd.x - Qd.x, Y = Pd.y - Qd.y, Z = Pd.z - Qd.z;
        const double R2 = fma(X, X, fma(Y, Y, Z * Z));
        const float Xf = Pf.x - Qf.x, Yf = Pf.y - Qf.y, Zf = Pf.z - Qf.z;
        const float R2f = fmaf(Xf, Xf, fmaf(Yf, Yf, Zf * Zf));
        const float pqf = Pf.w * Qf.w, sf = Pf.w + Qf.w;
        const bool asym = pqf * R2f >= (float)kBoysTmax * sf;
        // asymptotic (point-multipole) form for every lane; lanes below the switch overwrite it
        const double yv = rsqrt_from_seed(R2, rsqrt_approx(R2f));
        double base[L + 1];
        base[0] = keep ? yv : 0.0;
        if constexpr (L > 0) {
            const double ny2 = -(yv * yv);
            static_for<L>([&](auto N) {
                constexpr int n = decltype(N)::value;
                if constexpr (n == 0)
                    base[1] = base[0] * ny2;
                else
                    base[n + 1] = base[n] * (double(2 * n + 1) * ny2);
            });
        }
        if (!__all_sync(0xffffffffu, asym)) {
            if (!asym) {
                const Base64<L> t = fp64_table_base<L>(d.boys, Pd.w, Qd.w, __ldg(QRP + k), inv_aP, R2,
                                                       __fdividef(pqf, sf) * R2f);
#pragma unroll
                for (int n = 0; n <= L; ++n) base[n] = keep ? t.v[n] : 0.0;
            }
        }
        double R[NR];
        md_R<L, double>(R, base, X, Y, Z);
        hermite_bra<NP, NQ, double>(R, DQ, JP);
        hermite_ket_stage<NP, NQ>(R, DP, kbuf, cnt, lane);
        if (lane == 0) kbuf.k[cnt] = k;
        if (++cnt == kBatch) {
            ketbuf_flush_scaled<NQ>(kbuf, cnt, QJ, (size_t)nQ, QRP, lane);
            cnt = 0;
        }
    }
    if (cnt > 0) ketbuf_flush_scaled<NQ>(kbuf, cnt, QJ, (size_t)nQ, QRP, lane);
    if (valid) {
#pragma unroll
        for (int i = 0; i < NP; ++i) atomicAdd(d.pp_Jh[LP] + (size_t)i * nP + Pl, JP[i] * aP);
    }
}

// The ket-side field of a batch of nk consecutive kets of the FP32 core: the lane owning a (ket,
// component) slot sums its column over the 32 bra lanes, multiplies by the ket's scale k = k_hi + k_lo
// (kept as a float pair so that its rounding does not repeat in every partner's contribution) and adds
// the result to the FP64 accumulator.
template <int NQ, int RQ>
__device__ __forceinline__ void ketbuf_flush_rec(const KetBuf32& kb, int nk, int k0, double* __restrict__ QJ,
                                                 size_t nQ, const float* __restrict__ QR, int lane)
{
    __syncwarp();
    if (lane < nk * NQ) {
        float sum = 0.0f;
#pragma unroll 8
        for (int r = 0; r < 32; ++r) sum += kb.v[r * kKetBufLd + lane];
        const int k = k0 + lane / NQ;
        const float2 kk = __ldg(reinterpret_cast<const float2*>(QR + (size_t)k * RQ + 4));
        atomicAdd(QJ + (size_t)(lane % NQ) * nQ + k, f2d(fmaf(sum, kk.y, sum * kk.x)));
    }
    __syncwarp();
}

// NQ consecutive floats from 16-byte aligned p (vector loads; padding beyond NQ is not used)
template <int NQ>
__device__ __forceinline__ void load_weights(const float* __restrict__ p, float* u)
{
    static_for<(NQ + 3) / 4>([&](auto V) {
        constexpr int v = decltype(V)::value;
        const float4 w = __ldg(reinterpret_cast<const float4*>(p) + v);
        if constexpr (4 * v + 0 < NQ) u[4 * v + 0] = w.x;
        if constexpr (4 * v + 1 < NQ) u[4 * v + 1] = w.y;
        if constexpr (4 * v + 2 < NQ) u[4 * v + 2] = w.z;
        if constexpr (4 * v + 3 < NQ) u[4 * v + 3] = w.w;
    });
}

// Mixed-precision core for the register classes (L_P + L_Q <= 4), on the weights u = p^{-1/2} (D_P - D_P^ref)
// of the FP32 records.  With R' the Hermite integrals of the unit-normalised Coulomb kernel
// (R = (sqrt(pi)/2) p^{-1/2} q^{-1/2} R'; R' of the point multipoles, derivatives of 1/R, beyond the
// asymptotic switch), J_P = k_P sum_Q R' u_Q and J_Q = k_Q sum_P R' u_P with k = (sqrt(pi)/2) p^{-1/2}.
// FP32 geometry (each bra centre relative to the ket fragment's first atom, rounded once per tile),
// Boys function, recursion and contractions; 1/R by rsqrt_nr; the bra field in a two-sum float pair
// folded at the end of every ket batch; k applied as a float pair; all global accumulation FP64.
// The records' weights carry each fragment's total charge exactly to one rounding (k_fp32_charge_fix),
// and rounding the scale factors as float pairs keeps per-pair roundings from repeating coherently
// over all partners: what remains is the per-quartet FP32 rounding.  Schwarz screening is evaluated
// only in tiles whose smallest bra factor times the partner class's smallest ket factor is below tau
// (SCREEN).  B bra pairs per lane (positions tl.y + lane and tl.y + 32 + lane for B = 2): the per-ket
// work (record loads, loop, votes, staging of the ket-side field) is shared by B quartets.
template <int LP, int LQ, int B, bool SCREEN>
__device__ __forceinline__ void jtile_fp32_sp(const Dev& d, const int x, const int y, const int pos0, const int kb,
                                              const int ke, const float tau, const int lane, const KetBuf32& kbuf)
{
    constexpr int NP = nh(LP), NQ = nh(LQ), L = LP + LQ, NR = nh(LP + LQ);
    constexpr int kBatch = 32 / NQ;
    constexpr int RP = rec32_len(LP), RQ = rec32_len(LQ);
    constexpr float kTsw = L <= 2 ? kFp32SwitchLow : kFp32SwitchHigh;
    const int bra_end = d.frag_pp0[x * kClasses + LP] + d.frag_npp[x * kClasses + LP];
    const int kc = d.frag_pp0[y * kClasses + LQ];
    const int k0 = kc + kb;
    const int k1 = kc + min(ke, d.frag_npp[y * kClasses + LQ]);
    if (k0 >= k1) return;  // a ket chunk beyond the partner's range
    const double* ay = d.atom_xyz + 3 * d.frag_atom0[y];
    float px[B], py[B], pz[B], pP[B], qP[B], kh[B], kl[B], uP[B][NP], JP[B][NP], Jhi[B][NP], Jlo[B][NP];
    int Pl[B];
    bool valid[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int pos = pos0 + 32 * b + lane;
        valid[b] = pos < bra_end;
        Pl[b] = d.pp_perm[LP][valid[b] ? pos : pos0];
        const float* __restrict__ brec = d.pp_rec32[LP] + (size_t)Pl[b] * RP;
        const float4 b1 = __ldg(reinterpret_cast<const float4*>(brec) + 1);
        const double4_32a Pd = d.pp_P[LP][Pl[b]];
        px[b] = (float)(Pd.x - ay[0]);
        py[b] = (float)(Pd.y - ay[1]);
        pz[b] = (float)(Pd.z - ay[2]);
        pP[b] = (float)Pd.w;
        qP[b] = b1.z;
        kh[b] = b1.x;
        kl[b] = b1.y;
        load_weights<NP>(brec + 8, uP[b]);
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            if (!valid[b]) uP[b][i] = 0.0f;
            JP[b][i] = Jhi[b][i] = Jlo[b][i] = 0.0f;
        }
    }
    const float* __restrict__ QR = d.pp_rec32[LQ];
    double* __restrict__ QJ = d.pp_Jh[LQ];
    const size_t nQ = (size_t)d.n_pp[LQ];
    for (int kq = k0; kq < k1; kq += kBatch) {
        const int nk = min(kBatch, k1 - kq);
        const float* __restrict__ qr = QR + (size_t)kq * RQ;
        // without screening the next ket's record is loaded while the current one is in use
        float4 q0n;
        float uQn[NQ];
        if constexpr (!SCREEN) {
            q0n = __ldg(reinterpret_cast<const float4*>(qr));
            load_weights<NQ>(qr + 8, uQn);
        }
        for (int c = 0; c < nk; ++c, qr += RQ) {
            bool keep[B];
#pragma unroll
            for (int b = 0; b < B; ++b) keep[b] = true;
            if constexpr (SCREEN) {
                const float qQ = __ldg(qr + 6);
                bool any = false;
#pragma unroll
                for (int b = 0; b < B; ++b) {
                    keep[b] = qP[b] * qQ >= tau;
                    any = any || keep[b];
                }
                if (!__any_sync(0xffffffffu, any)) {
                    float* row = kbuf.v + lane * kKetBufLd + c * NQ;
#pragma unroll
                    for (int j = 0; j < NQ; ++j) row[j] = 0.0f;
                    continue;
                }
            }
            float4 q0;
            float uQ[NQ];
            if constexpr (SCREEN) {
                q0 = __ldg(reinterpret_cast<const float4*>(qr));
                load_weights<NQ>(qr + 8, uQ);
            } else {
                q0 = q0n;
#pragma unroll
                for (int j = 0; j < NQ; ++j) uQ[j] = uQn[j];
                if (c + 1 < nk) {
                    q0n = __ldg(reinterpret_cast<const float4*>(qr + RQ));
                    load_weights<NQ>(qr + RQ + 8, uQn);
                }
            }
            float stage[NQ];
#pragma unroll
            for (int j = 0; j < NQ; ++j) stage[j] = 0.0f;
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const float X = px[b] - q0.x, Y = py[b] - q0.y, Z = pz[b] - q0.z;
                const float R2 = fmaf(X, X, fmaf(Y, Y, Z * Z));
                const float pq = pP[b] * q0.w, sq = pP[b] + q0.w;
                const bool asym = pq * R2 >= kTsw * sq;
                // point-multipole form for every lane; lanes below the switch overwrite it
                float yv = rsqrt_nr(R2);
                if constexpr (SCREEN) {
                    if (!keep[b]) yv = 0.0f;
                }
                float base[L + 1];
                base[0] = yv;
                if constexpr (L > 0) {
                    const float ny2 = -(yv * yv);
                    static_for<L>([&](auto N) {
                        constexpr int n = decltype(N)::value;
                        if constexpr (n == 0)
                            base[1] = base[0] * ny2;
                        else
                            base[n + 1] = base[n] * (float(2 * n + 1) * ny2);
                    });
                }
                if (!__all_sync(0xffffffffu, asym)) {
                    if (!asym) {
                        const Base32<L> t = fp32_table_base<L>(d.boys32, pq, sq, R2);
#pragma unroll
                        for (int n = 0; n <= L; ++n) base[n] = (SCREEN && !keep[b]) ? 0.0f : t.v[n];
                    }
                }
                float R[NR];
                md_R<L, float>(R, base, X, Y, Z);
                hermite_bra<NP, NQ, float>(R, uQ, JP[b]);
                // this bra's share of the ket-side field, (-1)^{|j|} sum_i R[i + j] u_P[i]
                static_for<NQ>([&](auto Jc) {
                    constexpr TUV bq = htuv(decltype(Jc)::value);
                    float sum = 0.0f;
                    static_for<NP>([&](auto I) {
                        constexpr TUV a = htuv(decltype(I)::value);
                        sum = fmaf(R[hidx(a.t + bq.t, a.u + bq.u, a.v + bq.v)], uP[b][decltype(I)::value], sum);
                    });
                    if constexpr (((bq.t + bq.u + bq.v) & 1) != 0)
                        stage[decltype(Jc)::value] -= sum;
                    else
                        stage[decltype(Jc)::value] += sum;
                });
            }
            float* row = kbuf.v + lane * kKetBufLd + c * NQ;
#pragma unroll
            for (int j = 0; j < NQ; ++j) row[j] = stage[j];
        }
        ketbuf_flush_rec<NQ, RQ>(kbuf, nk, kq, QJ, nQ, QR, lane);
#pragma unroll
        for (int b = 0; b < B; ++b)
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                two_sum_acc(Jhi[b][i], Jlo[b][i], JP[b][i]);
                JP[b][i] = 0.0f;
            }
    }
#pragma unroll
    for (int b = 0; b < B; ++b) {
        if (!valid[b]) continue;
        // (Jhi + Jlo) (k_hi + k_lo) as a float pair: Jhi k_hi exactly (FMA residual) plus the cross terms
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            const float hi = Jhi[b][i] * kh[b];
            const float lo = fmaf(Jhi[b][i], kh[b], -hi) + fmaf(Jhi[b][i], kl[b], Jlo[b][i] * kh[b]);
            double* dst = d.pp_Jh[LP] + (size_t)i * d.n_pp[LP] + Pl[b];
            atomicAdd(dst, f2d(hi));
            atomicAdd(dst, f2d(lo));
        }
    }
}

// FP32-core tile of a register class (L_P + L_Q <= 4, d-shell classes included) on the records with B
// bra pairs per lane, the Schwarz test only where some quartet of the tile can fail it.
template <int LP, int LQ, int B = 1>
__device__ __forceinline__ void jtile_fp32(const Dev& d, const int2 tl, const int kb, const int ke, const float tau,
                                           const int lane, const KetBuf32& kbuf)
{
    const int pr = tl.x >> 1;
    const int x = (tl.x & 1) ? d.pair_y[pr] : d.pair_x[pr];
    const int y = (tl.x & 1) ? d.pair_x[pr] : d.pair_y[pr];
    const int bra_end = d.frag_pp0[x * kClasses + LP] + d.frag_npp[x * kClasses + LP];
    float qmin = 3.0e38f;
#pragma unroll
    for (int b = 0; b < B; ++b)
        if (tl.y + 32 * b + lane < bra_end) qmin = fminf(qmin, d.pp_Q[LP][d.pp_perm[LP][tl.y + 32 * b + lane]]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) qmin = fminf(qmin, __shfl_xor_sync(0xffffffffu, qmin, o));
    if (qmin * __ldg(d.fc_qmin + y * kClasses + LQ) < tau)
        jtile_fp32_sp<LP, LQ, B, true>(d, x, y, tl.y, kb, ke, tau, lane, kbuf);
    else
        jtile_fp32_sp<LP, LQ, B, false>(d, x, y, tl.y, kb, ke, tau, lane, kbuf);
}

// Ket chunk c of nchunk of a per-class launch: partner offsets [c chunk, (c + 1) chunk), or the whole
// range when chunk = 0.
__device__ __forceinline__ void ket_chunk_range(int c, int chunk, int& kb, int& ke)
{
    kb = chunk > 0 ? c * chunk : 0;
    ke = chunk > 0 ? kb + chunk : INT_MAX;
}

// One warp per (tile, ket chunk), one launch per class pair.
template <int LP, int LQ>
__global__ void __launch_bounds__(128) k_jengine(Dev d, const int2* __restrict__ tiles, int n_tiles, float tau,
                                                 int chunk, int nchunk)
{
    __shared__ double kv[4 * kKetBufWarp];
    __shared__ int kk[4 * 32];
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int unit = warp / nchunk;
    if (unit >= n_tiles) return;
    int kb, ke;
    ket_chunk_range(warp - unit * nchunk, chunk, kb, ke);
    const int w = threadIdx.x >> 5;
    jtile_fp64<LP, LQ>(d, tiles[unit], kb, ke, tau, threadIdx.x & 31, KetBuf{kv + w * kKetBufWarp, kk + w * 32});
}

// FP32 core, one launch per class pair.  For L_P <= 1 a warp takes two consecutive tiles: when they
// cover the same fragment pair (64 consecutive bra positions) it runs them as one tile with two bra
// pairs per lane, else one after the other.
template <int LP, int LQ>
__global__ void __launch_bounds__(128) k_jengine32(Dev d, const int2* __restrict__ tiles, int n_tiles, float tau,
                                                   int chunk, int nchunk)
{
    __shared__ float kv[4 * kKetBufWarp];
    __shared__ int kk[4 * 32];
    constexpr int kPer = LP <= 1 ? 2 : 1;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int unit = warp / nchunk;
    const int t0 = unit * kPer;
    if (t0 >= n_tiles) return;
    int kb, ke;
    ket_chunk_range(warp - unit * nchunk, chunk, kb, ke);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const KetBuf32 kbuf{kv + w * kKetBufWarp, kk + w * 32};
    const int2 a = tiles[t0];
    if constexpr (kPer == 2) {
        if (t0 + 1 < n_tiles) {
            const int2 b = tiles[t0 + 1];
            if (b.x == a.x && b.y == a.y + 32) {
                jtile_fp32<LP, LQ, 2>(d, a, kb, ke, tau, lane, kbuf);
                return;
            }
            jtile_fp32<LP, LQ>(d, a, kb, ke, tau, lane, kbuf);
            jtile_fp32<LP, LQ>(d, b, kb, ke, tau, lane, kbuf);
            return;
        }
    }
    jtile_fp32<LP, LQ>(d, a, kb, ke, tau, lane, kbuf);
}

// ------------------------------------------------------------------------------------------ persistent
// Persistent J-engine: the grid is sized to the resident capacity of the GPU and every warp takes
// work items from a cost-sorted queue (one atomic per item) until it is empty, so quartet classes
// of all fragment pairs (of uneven size and mixed angular momentum) share one launch and the
// longest items start first.  An item is one 32-bra-pair tile against a chunk of the partner's
// ket pairs (JItem encoding in internal.hpp).  MODE 0: FP64 core, 1: FP32 core.  SPD adds the
// register classes with a d-shell pair (L_P = 3, 4; L_P + L_Q <= 4), whose larger register
// footprint would otherwise lower the occupancy of the s/p classes.
template <int MODE, int LP, int LQ>
__device__ __forceinline__ void jtile(const Dev& d, int2 tl, int kb, int ke, float tau, int lane, const KetBuf& kbuf,
                                      const KetBuf32& kbuf32)
{
    if constexpr (MODE == 0)
        jtile_fp64<LP, LQ>(d, tl, kb, ke, tau, lane, kbuf);
    else
        jtile_fp32<LP, LQ>(d, tl, kb, ke, tau, lane, kbuf32);
}

template <int MODE, bool SPD>
__global__ void __launch_bounds__(128) k_jengine_persistent(Dev d, const int4* __restrict__ items, int n_items,
                                                            int* __restrict__ next, float tau)
{
    // the ket-side field is staged in shared memory (one buffer per warp, of the core's type)
    __shared__ double kv[MODE == 0 ? 4 * kKetBufWarp : 1];
    __shared__ float kv32[MODE == 0 ? 1 : 4 * kKetBufWarp];
    __shared__ int kk[4 * 32];
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const KetBuf kbuf{kv + (MODE == 0 ? w * kKetBufWarp : 0), kk + w * 32};
    const KetBuf32 kbuf32{kv32 + (MODE == 0 ? 0 : w * kKetBufWarp), kk + w * 32};
    for (;;) {
        int i = 0;
        if (lane == 0) i = atomicAdd(next, 1);
        i = __shfl_sync(0xffffffffu, i, 0);
        if (i >= n_items) return;
        const int4 it = items[i];
        const int2 tl = make_int2(it.x, it.y);
        const int kb = it.z, ke = jitem_ket_end(it);
        switch (jitem_class(it)) {
            case 0 * kClasses + 0: jtile<MODE, 0, 0>(d, tl, kb, ke, tau, lane, kbuf, kbuf32); break;
            case 1 * kClasses + 0: jtile<MODE, 1, 0>(d, tl, kb, ke, tau, lane, kbuf, kbuf32); break;
            case 1 * kClasses + 1: jtile<MODE, 1, 1>(d, tl, kb, ke, tau, lane, kbuf, kbuf32); break;
            case 2 * kClasses + 0: jtile<MODE, 2, 0>(d, tl, kb, ke, tau, lane, kbuf, kbuf32); break;
            case 2 * kClasses + 1: jtile<MODE, 2, 1>(d, tl, kb, ke, tau, lane, kbuf, kbuf32); break;
            case 2 * kClasses + 2: jtile<MODE, 2, 2>(d, tl, kb, ke, tau, lane, kbuf, kbuf32); break;
            case 3 * kClasses + 0: if constexpr (SPD) jtile<MODE, 3, 0>(d, tl, kb, ke, tau, lane, kbuf, kbuf32); break;
            case 3 * kClasses + 1: if constexpr (SPD) jtile<MODE, 3, 1>(d, tl, kb, ke, tau, lane, kbuf, kbuf32); break;
            case 4 * kClasses + 0: if constexpr (SPD) jtile<MODE, 4, 0>(d, tl, kb, ke, tau, lane, kbuf, kbuf32); break;
            default: break;
        }
    }
}

static const void* persistent_kernel(int mode, bool spd)
{
    if (mode == 0) return spd ? (const void*)k_jengine_persistent<0, true> : (const void*)k_jengine_persistent<0, false>;
    return spd ? (const void*)k_jengine_persistent<1, true> : (const void*)k_jengine_persistent<1, false>;
}

cudaError_t jengine_persistent_grid(int mode, bool spd, int* blocks_per_sm)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, persistent_kernel(mode, spd), 128, 0);
}

cudaError_t launch_jengine_persistent(const Dev& d, int mode, bool spd, const JQueue& q, float tau, cudaStream_t s)
{
    if (q.n <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(q.next, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    const int blocks = std::max(1, std::min(q.grid, (q.n + 3) / 4));
    if (mode == 0) {
        if (spd) k_jengine_persistent<0, true><<<blocks, 128, 0, s>>>(d, q.items, q.n, q.next, tau);
        else k_jengine_persistent<0, false><<<blocks, 128, 0, s>>>(d, q.items, q.n, q.next, tau);
    } else {
        if (spd) k_jengine_persistent<1, true><<<blocks, 128, 0, s>>>(d, q.items, q.n, q.next, tau);
        else k_jengine_persistent<1, false><<<blocks, 128, 0, s>>>(d, q.items, q.n, q.next, tau);
    }
    note_launches(1);
    return cudaGetLastError();
}

// chunk > 0: every tile is cut into nchunk ket chunks of chunk partner pairs (one warp each)
template <int LP, int LQ>
static void launch_one(const Dev& d, const int2* t, int n, float tau, int fp32, cudaStream_t s, int chunk = 0,
                       int nchunk = 1)
{
    if (n <= 0) return;
    if (chunk <= 0) nchunk = 1;
    const int warps_per_block = 4;
    if (fp32) {
        const int per = LP <= 1 ? 2 : 1;  // tiles per warp of the FP32 core (see k_jengine32)
        const long long warps = (long long)((n + per - 1) / per) * nchunk;
        k_jengine32<LP, LQ><<<(unsigned)((warps + warps_per_block - 1) / warps_per_block), 32 * warps_per_block, 0,
                              s>>>(d, t, n, tau, chunk, nchunk);
    } else {
        const long long warps = (long long)n * nchunk;
        k_jengine<LP, LQ><<<(unsigned)((warps + warps_per_block - 1) / warps_per_block), 32 * warps_per_block, 0,
                            s>>>(d, t, n, tau, chunk, nchunk);
    }
    note_launches(1);
}

// One class pair's kernel on stream s (mode 0 FP64, 1 FP32, 2 float-float for L_P <= 2): the plans
// that run the class kernels concurrently on forked streams launch them one by one.
cudaError_t launch_jengine_class(const Dev& d, int LP, int LQ, const int2* t, int n, float tau, int mode, cudaStream_t s,
                                 int chunk, int nchunk)
{
    if (n <= 0) return cudaSuccess;
    if (LP + LQ >= 5) return launch_jengine_big_class(d, LP, LQ, t, n, tau, mode == 1 ? 1 : 0, s);
    if (mode == 2 && LP <= 2) return launch_jengine_df_class(d, LP, LQ, t, n, tau, s);
    const int fp32 = mode == 1 ? 1 : 0;
    switch (LP * kClasses + LQ) {
        case 0 * kClasses + 0: launch_one<0, 0>(d, t, n, tau, fp32, s, chunk, nchunk); break;
        case 1 * kClasses + 0: launch_one<1, 0>(d, t, n, tau, fp32, s, chunk, nchunk); break;
        case 1 * kClasses + 1: launch_one<1, 1>(d, t, n, tau, fp32, s, chunk, nchunk); break;
        case 2 * kClasses + 0: launch_one<2, 0>(d, t, n, tau, fp32, s, chunk, nchunk); break;
        case 2 * kClasses + 1: launch_one<2, 1>(d, t, n, tau, fp32, s, chunk, nchunk); break;
        case 2 * kClasses + 2: launch_one<2, 2>(d, t, n, tau, fp32, s, chunk, nchunk); break;
        case 3 * kClasses + 0: launch_one<3, 0>(d, t, n, tau, fp32, s, chunk, nchunk); break;
        case 3 * kClasses + 1: launch_one<3, 1>(d, t, n, tau, fp32, s, chunk, nchunk); break;
        case 4 * kClasses + 0: launch_one<4, 0>(d, t, n, tau, fp32, s, chunk, nchunk); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_jengine(const Dev& d, const int2* tiles[kClasses][kClasses], const int* n_tiles, double tau,
                           int mode, cudaStream_t s)
{
    const float ft = (float)tau;
    const int fp32 = mode == 1 ? 1 : 0;
#define FEF_J(LP, LQ) launch_one<LP, LQ>(d, tiles[LP][LQ], n_tiles[LP * kClasses + LQ], ft, fp32, s)
    if (mode == 2) {
        cudaError_t e = launch_jengine_df(d, tiles, n_tiles, ft, s);
        if (e != cudaSuccess) return e;
    } else {
        FEF_J(0, 0); FEF_J(1, 0); FEF_J(1, 1); FEF_J(2, 0); FEF_J(2, 1); FEF_J(2, 2);
    }
    FEF_J(3, 0); FEF_J(3, 1); FEF_J(4, 0);
#undef FEF_J
    return launch_jengine_big(d, tiles, n_tiles, ft, fp32, s);  // classes with L_P + L_Q >= 5
}

// FP32-core records (layout: rec32_len in internal.hpp), one thread per primitive pair of class L:
// (P - anchor, p) | (k_hi, k_lo, Q, 0) | u = p^{-1/2} (D_P - D_P^ref) rounded to FP32; resid[g] keeps
// u[0] - float(u[0]) for the charge fix below.
__global__ void k_fp32_records(Dev d, int L, const double* __restrict__ ref, double* __restrict__ resid)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = d.n_pp[L];
    if (g >= n) return;
    const int NH = nh(L), RL = rec32_len(L);
    float* r = d.pp_rec32[L] + (size_t)g * RL;
    const double rp = d.pp_rp[L][g];
    const double k = kSqrtPiHalf * rp;
    const float khi = (float)k;
    reinterpret_cast<float4*>(r)[0] = d.pp_Pr[L][g];
    reinterpret_cast<float4*>(r)[1] = make_float4(khi, (float)(k - (double)khi), d.pp_Q[L][g], 0.0f);
    for (int i = 0; i < NH; ++i) {
        const size_t o = (size_t)i * n + g;
        const double u = rp * (d.pp_Dh[L][o] - (ref ? ref[o] : 0.0));
        const float uh = (float)u;
        r[8 + i] = uh;
        if (i == 0) resid[g] = u - (double)uh;
    }
    for (int i = NH; i < RL - 8; ++i) r[8 + i] = 0.0f;
}

// Charge-conserving rounding of the FP32 weights, one block per fragment for class L: the sum of the
// roundings of u[0] over the fragment's class range is moved onto its element of smallest |u[0]|, so
// that the FP32 weights sum to the exact total to within one rounding of that element.  Every
// partner's quartets reuse these weights, so an uncorrected sum of roundings would act as a spurious
// charge in the field of all neighbours at once (a coherent, not a random, error).
__global__ void k_fp32_charge_fix(Dev d, int L, const double* __restrict__ resid)
{
    const int x = blockIdx.x;
    const int g0 = d.frag_pp0[x * kClasses + L], m = d.frag_npp[x * kClasses + L];
    if (m == 0) return;
    const int RL = rec32_len(L);
    float* rec = d.pp_rec32[L];
    double sum = 0.0;
    float best = 3.0e38f;
    int arg = g0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const int g = g0 + i;
        sum += resid[g];
        const float a = fabsf(rec[(size_t)g * RL + 8]);
        if (a < best || (a == best && g < arg)) {
            best = a;
            arg = g;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
        const float b2 = __shfl_xor_sync(0xffffffffu, best, o);
        const int a2 = __shfl_xor_sync(0xffffffffu, arg, o);
        if (b2 < best || (b2 == best && a2 < arg)) {
            best = b2;
            arg = a2;
        }
    }
    __shared__ double s_sum[32];
    __shared__ float s_best[32];
    __shared__ int s_arg[32];
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s_sum[w] = sum;
        s_best[w] = best;
        s_arg[w] = arg;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        float b = 3.0e38f;
        int a = g0;
        for (int i = 0; i < nw; ++i) {
            t += s_sum[i];
            if (s_best[i] < b || (s_best[i] == b && s_arg[i] < a)) {
                b = s_best[i];
                a = s_arg[i];
            }
        }
        float* u0 = rec + (size_t)a * RL + 8;
        *u0 = (float)((double)*u0 + t);
    }
}

cudaError_t launch_fp32_records(const Dev& d, double* const Dh_ref[kClasses], double* resid, cudaStream_t s)
{
    for (int L = 0; L < kClasses; ++L) {
        if (d.n_pp[L] == 0) continue;
        k_fp32_records<<<(d.n_pp[L] + 127) / 128, 128, 0, s>>>(d, L, Dh_ref[L], resid);
        k_fp32_charge_fix<<<d.n_frag, 128, 0, s>>>(d, L, resid);
        note_launches(2);
    }
    return cudaGetLastError();
}

// Smallest Schwarz factor of every fragment's primitive pairs of each class (FLT_MAX-like when the
// class is empty): one warp per (fragment, class).
__global__ void k_class_qmin(Dev d, float* qmin)
{
    const int x = blockIdx.x, L = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g0 = d.frag_pp0[x * kClasses + L], m = d.frag_npp[x * kClasses + L];
    float q = 3.0e38f;
    for (int i = lane; i < m; i += 32) q = fminf(q, d.pp_Q[L][g0 + i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q = fminf(q, __shfl_xor_sync(0xffffffffu, q, o));
    if (lane == 0) qmin[x * kClasses + L] = q;
}

cudaError_t launch_class_qmin(const Dev& d, float* qmin, cudaStream_t s)
{
    k_class_qmin<<<d.n_frag, 32 * kClasses, 0, s>>>(d, qmin);
    note_launches(1);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------ back-transform
// J^x_{mu nu} = (c/p) sum_{P in shell pair of (mu, nu)} sum_tuv E^{mu nu}_tuv(P) Jh_P[tuv], scaled to
// normalised AOs.  One warp per shell pair (a <= b) of every fragment: each lane takes primitive pairs
// of the shell pair and forms their Hermite expansion coefficients once for all Cartesian component
// pairs (compile-time l_a, l_b), the warp sums over the primitive pairs by a butterfly (a fixed order,
// so the result is reproducible), and lane 0 writes J[mu][nu] and J[nu][mu].
template <int LA, int LB>
__device__ __forceinline__ void back_transform_pair(const Dev& d, int sp, int lane, double* __restrict__ J)
{
    constexpr int NA = ncart(LA), NB = ncart(LB), L = LA + LB, NH = nh(LA + LB);
    const int s1 = d.sp_a[sp], s2 = d.sp_b[sp];
    const int x = frag_of_shellpair(d, sp);
    const double* A = d.atom_xyz + 3 * d.sh_atom[s1];
    const double* B = d.atom_xyz + 3 * d.sh_atom[s2];
    const int npp = d.n_pp[L];
    const int np = d.sh_np[s1] * d.sh_np[s2];
    const int g0 = d.sp_pp0[sp];
    double acc[NA * NB];
#pragma unroll
    for (int e = 0; e < NA * NB; ++e) acc[e] = 0.0;
    for (int k = lane; k < np; k += 32) {
        const int g = g0 + k;
        const double4_32a P = d.pp_P[L][g];
        double E[3][3][3][5];
        md_E1(LA, LB, P.w, P.x - A[0], P.x - B[0], E[0]);
        md_E1(LA, LB, P.w, P.y - A[1], P.y - B[1], E[1]);
        md_E1(LA, LB, P.w, P.z - A[2], P.z - B[2], E[2]);
        double Jh[NH];
#pragma unroll
        for (int h = 0; h < NH; ++h) Jh[h] = d.pp_Jh[L][(size_t)h * npp + g];
        const double sc = d.pp_K[L][g] * kSqrt2Pi52 / P.w;
#pragma unroll
        for (int ia = 0; ia < NA; ++ia) {
            int ax, ay, az;
            cart_of(LA, ia, ax, ay, az);
#pragma unroll
            for (int ib = 0; ib < NB; ++ib) {
                int bx, by, bz;
                cart_of(LB, ib, bx, by, bz);
                double v = 0.0;
#pragma unroll
                for (int t = 0; t <= L; ++t)
#pragma unroll
                    for (int u = 0; u <= L - t; ++u)
#pragma unroll
                        for (int w = 0; w <= L - t - u; ++w)
                            if (t <= ax + bx && u <= ay + by && w <= az + bz)
                                v += E[0][ax][bx][t] * E[1][ay][by][u] * E[2][az][bz][w] * Jh[hidx(t, u, w)];
                acc[ia * NB + ib] = fma(v, sc, acc[ia * NB + ib]);
            }
        }
    }
#pragma unroll
    for (int e = 0; e < NA * NB; ++e)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[e] += __shfl_xor_sync(0xffffffffu, acc[e], o);
    if (lane == 0) {
        const int n = d.frag_nao[x], ao0 = d.frag_ao0[x];
        const int mu0 = d.sh_ao[s1], nu0 = d.sh_ao[s2];
        double* Jx = J + d.frag_moff[x];
#pragma unroll
        for (int ia = 0; ia < NA; ++ia)
#pragma unroll
            for (int ib = 0; ib < NB; ++ib) {
                const int mu = mu0 + ia, nu = nu0 + ib;
                const double v = acc[ia * NB + ib] * d.ao_scale[ao0 + mu] * d.ao_scale[ao0 + nu];
                Jx[mu * n + nu] = v;
                Jx[nu * n + mu] = v;
            }
    }
}

// Shell pairs of s and p shells, and (second kernel, so that the s/p one keeps its small register
// footprint) the pairs with a d shell.
__global__ void __launch_bounds__(128) k_back_transform_sp(Dev d, double* J)
{
    const int sp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (sp >= d.n_sp) return;
    switch (d.sh_l[d.sp_a[sp]] * 3 + d.sh_l[d.sp_b[sp]]) {
        case 0: back_transform_pair<0, 0>(d, sp, lane, J); break;
        case 1: back_transform_pair<0, 1>(d, sp, lane, J); break;
        case 3: back_transform_pair<1, 0>(d, sp, lane, J); break;
        case 4: back_transform_pair<1, 1>(d, sp, lane, J); break;
        default: break;
    }
}

__global__ void __launch_bounds__(128) k_back_transform_d(Dev d, double* J)
{
    const int sp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (sp >= d.n_sp) return;
    switch (d.sh_l[d.sp_a[sp]] * 3 + d.sh_l[d.sp_b[sp]]) {
        case 2: back_transform_pair<0, 2>(d, sp, lane, J); break;
        case 5: back_transform_pair<1, 2>(d, sp, lane, J); break;
        case 6: back_transform_pair<2, 0>(d, sp, lane, J); break;
        case 7: back_transform_pair<2, 1>(d, sp, lane, J); break;
        case 8: back_transform_pair<2, 2>(d, sp, lane, J); break;
        default: break;
    }
}

cudaError_t launch_back_transform(const Dev& d, double* J, cudaStream_t s)
{
    if (d.n_sp <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)(((int64_t)d.n_sp * 32 + 127) / 128);
    k_back_transform_sp<<<blocks, 128, 0, s>>>(d, J);
    note_launches(1);
    if (d.max_l >= 2) {
        k_back_transform_d<<<blocks, 128, 0, s>>>(d, J);
        note_launches(1);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------ Fock
// F^x = h^x + G[D^x] + V_env^x + J_env^x with G = C D (C: packed transposed Coulomb-minus-half-
// exchange tensor, see setup.cu), plus E_int[x] = tr[D (h + G/2)] + E_nn(x) and tr[D omega]
// (omega = V_env + J_env).  One block per fragment; thread per packed row pq = (mu <= nu).
__global__ void k_fock_assemble(Dev d, const double* h, const double* Venv, const double* Jenv, const double* eric,
                                const double* D, double* F, double* omega, const double* e_nn, double* E_int,
                                double* trV, double* trJ)
{
    int x = blockIdx.x;
    int n = d.frag_nao[x];
    int np = n * (n + 1) / 2;
    const double* C = eric + d.frag_coff[x];
    const double* Dx = D + d.frag_moff[x];
    extern __shared__ double dpk[];  // packed D_rs
    for (int rs = threadIdx.x; rs < np; rs += blockDim.x) {
        int la = 0, r = rs;
        while (r >= n - la) { r -= n - la; ++la; }
        dpk[rs] = Dx[la * n + la + r];
    }
    __syncthreads();
    double eint = 0.0, ev = 0.0, ej = 0.0;
    for (int pq = threadIdx.x; pq < np; pq += blockDim.x) {
        int mu = 0, r = pq;
        while (r >= n - mu) { r -= n - mu; ++mu; }
        int nu = mu + r;
        double g = 0.0;
        for (int rs = 0; rs < np; ++rs) g = fma(C[(size_t)rs * np + pq], dpk[rs], g);
        const double w = (mu == nu) ? 1.0 : 2.0;
        for (int k = 0; k < (mu == nu ? 1 : 2); ++k) {
            int64_t o = d.frag_moff[x] + (k == 0 ? mu * n + nu : nu * n + mu);
            double om = (Venv ? Venv[o] : 0.0) + (Jenv ? Jenv[o] : 0.0);
            if (F) F[o] = h[o] + g + om;
            if (omega) omega[o] = om;
        }
        int64_t o = d.frag_moff[x] + mu * n + nu;
        const double dw = w * Dx[mu * n + nu];
        eint += dw * (h[o] + 0.5 * g);
        ev += dw * (Venv ? Venv[o] : 0.0);
        ej += dw * (Jenv ? Jenv[o] : 0.0);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        eint += __shfl_xor_sync(0xffffffffu, eint, o);
        ev += __shfl_xor_sync(0xffffffffu, ev, o);
        ej += __shfl_xor_sync(0xffffffffu, ej, o);
    }
    __shared__ double r1[32], r2[32], r3[32];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (lane == 0) {
        r1[warp] = eint;
        r2[warp] = ev;
        r3[warp] = ej;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0, c = 0.0;
        for (int w = 0; w < nw; ++w) {
            a += r1[w];
            b += r2[w];
            c += r3[w];
        }
        if (E_int) E_int[x] = a + e_nn[x];
        if (trV) trV[x] = b;
        if (trJ) trJ[x] = c;
    }
}

cudaError_t launch_fock_energy(const Dev& d, const double* h, const double* Venv, const double* Jenv,
                               const double* eric, const double* D, double* F, double* omega, const double* e_nn,
                               double* E_int, double* trV, double* trJ, cudaStream_t s)
{
    size_t smem = sizeof(double) * (size_t)d.max_nao * (d.max_nao + 1) / 2;  // packed density, <= 227 KB
    cudaError_t e = cudaFuncSetAttribute(k_fock_assemble, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_fock_assemble<<<d.n_frag, 256, smem, s>>>(d, h, Venv, Jenv, eric, D, F, omega, e_nn, E_int, trV, trJ);
    note_launches(1);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------ energies
// Pair energy E_xy = tr[D^x V^y] + tr[D^y V^x] + tr[D^x J[D^y]] + E_nn(x,y).  Summed over the
// neighbours y of x, sum_y tr[D^x V^y] = tr[D^x V_env^x] and sum_y tr[D^x J[D^y]] = tr[D^x J_env^x]
// (the accumulated fields), so only the attraction of x's nuclei on each neighbour's electrons is
// needed per pair:
//   E_frag[x] = E_int[x] + (1/2) (tr[D^x V_env] + sum_y tr[D^y V^x] + tr[D^x J_env] + sum_y E_nn(x,y)),
//   E_total = sum_x E_frag[x] = sum_x E_int[x] + sum_{pairs} E_xy.
__global__ void k_frag_energy(Dev d, const double* E_int, const double* trV, const double* trJ, const double* tr_xy,
                              const double* tr_yx, const double* e_nn, double* E_frag)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= d.n_frag) return;
    double e = trV[x] + trJ[x];
    for (int c = d.frag_nbr0[x]; c < d.frag_nbr0[x + 1]; ++c) {
        int p = d.nbr_pair[c];
        e += (d.pair_x[p] == x ? tr_yx[p] : tr_xy[p]) + e_nn[p];
    }
    E_frag[x] = E_int[x] + 0.5 * e;
}

__global__ void k_total_energy(Dev d, const double* E_frag, double* E_tot)
{
    __shared__ double red[256];
    double a = 0.0;
    for (int i = threadIdx.x; i < d.n_frag; i += blockDim.x) a += E_frag[i];
    red[threadIdx.x] = a;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *E_tot = red[0];
}

cudaError_t launch_energies(const Dev& d, const double* E_int, const double* trV, const double* trJ,
                            const double* tr_xy, const double* tr_yx, const double* e_nn_pair, double* E_frag,
                            double* E_tot, cudaStream_t s)
{
    k_frag_energy<<<(d.n_frag + 255) / 256, 256, 0, s>>>(d, E_int, trV, trJ, tr_xy, tr_yx, e_nn_pair, E_frag);
    note_launches(1);
    k_total_energy<<<1, 256, 0, s>>>(d, E_frag, E_tot);
    note_launches(1);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------ checks
__global__ void k_check_finite(const double* a, int64_t n, int* flag)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(a[i])) {
            atomicOr(flag, kErrNumeric);
            return;
        }
}

cudaError_t launch_check_finite(const double* a, int64_t n, int* flag, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    int blocks = (int)std::min<int64_t>((n + 255) / 256, 1024);
    k_check_finite<<<blocks, 256, 0, s>>>(a, n, flag);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace fef

namespace fef {
// Inter-fragment shell quartets (a<=b in x, c<=d in y, x<y) with Q_ab Q_cd >= tau, and their
// primitive quartets per Hermite class (L_ab, L_cd): one block per pair.  count[0] = shell
// quartets, count[1 + L_ab*kClasses + L_cd] = primitive quartets of that class.
__global__ void k_count_quartets(Dev d, double tau, unsigned long long* count)
{
    __shared__ unsigned long long cls[kClasses * kClasses];
    for (int i = threadIdx.x; i < kClasses * kClasses; i += blockDim.x) cls[i] = 0;
    __syncthreads();
    int pr = blockIdx.x;
    int x = d.pair_x[pr], y = d.pair_y[pr];
    int s0 = d.frag_sp0[x], ns = d.frag_sp0[x + 1] - s0;
    int t0 = d.frag_sp0[y], nt = d.frag_sp0[y + 1] - t0;
    unsigned long long c = 0;
    for (int w = threadIdx.x; w < ns * nt; w += blockDim.x) {
        int s1 = s0 + w / nt, s2 = t0 + w % nt;
        if (d.sp_Q[s1] * d.sp_Q[s2] >= tau) {
            ++c;
            unsigned long long np = (unsigned long long)d.sh_np[d.sp_a[s1]] * d.sh_np[d.sp_b[s1]] *
                                    d.sh_np[d.sp_a[s2]] * d.sh_np[d.sp_b[s2]];
            atomicAdd(&cls[d.sp_L[s1] * kClasses + d.sp_L[s2]], np);
        }
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(count, c);
    __syncthreads();
    for (int i = threadIdx.x; i < kClasses * kClasses; i += blockDim.x)
        if (cls[i]) atomicAdd(count + 1 + i, cls[i]);
}

cudaError_t launch_count_quartets(const Dev& d, double tau, unsigned long long* count, cudaStream_t s)
{
    if (d.n_pairs > 0) {
        k_count_quartets<<<d.n_pairs, 128, 0, s>>>(d, tau, count);
        note_launches(1);
    }
    return cudaGetLastError();
}
}  // namespace fef
