// Dimer second-order energy of the FEF cluster perturbation theory (paper, Eq. ED2 with the first-order
// dimer doubles of Eq. dimDoubles) for fragment pairs whose shells are s and p:
//   E_D2^{xy} = 4 sum_{ia in x, jb in y} (ia|jb)^2 / (eps_i + eps_j - eps_a - eps_b),
// i occupied and a virtual canonical orbitals of x (j, b of y).  The integrals come from the Hermite
// Gaussian expansion of the transition densities phi_i phi_a (McMurchie-Davidson), in the conventions of
// the FP64 J-engine (jengine.cu): with u^{ia}_P[tuv] = p^{-1/2} (c/p) K_P sum_{mu nu in P} w^{ia}_{mu nu}
// E^{mu nu}_{tuv}(P) the pre-scaled transition Hermite density of primitive pair P,
//   (ia|jb) = (sqrt(pi)/2) sum_{P in x, Q in y} sum_{tuv, t'u'v'} u^{ia}_P[tuv] (-1)^{t'+u'+v'} R'_{t+t',u+u',v+v'}(P, Q) u^{jb}_Q[t'u'v'],
// R' the unit-normalised Hermite Coulomb integrals (point multipoles beyond the Boys asymptotic switch).
// Work is split as in a J-engine with many densities: for each bra primitive pair P (one lane) the field
// G_P[tuv][jb] = sum_Q sum_{t'u'v'} (-1)^{|t'|} R'[tuv + t'u'v'] u^{jb}_Q[t'u'v'] of all the partner's
// transition densities, a block of jb per warp; then (ia|jb) = (sqrt(pi)/2) sum_{P, tuv} u^{ia}_P[tuv]
// G_P[tuv][jb] per pair.  The member with the smaller Hermite class of a class pair is the bra, so that
// the lane's accumulators stay in registers; the quartet set is the J-engine's (cutoff pairs, shell-level
// Schwarz screening).  No AO-basis integral block is formed.
#include <algorithm>
#include <climits>

#include "common.cuh"
#include "df64.cuh"
#include "internal.hpp"

namespace fef {

namespace {

// jb columns of G per lane and bra Hermite component for bra class L (register budget of the lane's field)
__host__ __device__ constexpr int ed2_cols(int L) { return L == 0 ? 40 : (L == 1 ? 10 : 4); }

// Transition Hermite densities of every fragment for class L: thread per (primitive pair g, ov pair k).
// U[uoff[x] + (hoff[x*5+L] + (g - pp0) nh(L) + h) n_ov(x) + k].
__global__ void k_ed2_transition(Dev d, int L, const double* __restrict__ C, const int* __restrict__ nmo,
                                 const int64_t* __restrict__ uoff, const int* __restrict__ hoff,
                                 const int* __restrict__ n_ov, int max_ov, double* __restrict__ U)
{
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int npp = d.n_pp[L];
    if (tid >= (int64_t)npp * max_ov) return;
    const int g = (int)(tid / max_ov), k = (int)(tid % max_ov);
    const int sp = d.pp_sp[L][g], ij = d.pp_ij[L][g];
    const int x = frag_of_shellpair(d, sp);
    const int nov = n_ov[x];
    if (k >= nov) return;
    const int n = d.frag_nao[x], no = d.frag_nocc[x], nv = nmo[x] - no;
    const int i = k / nv, a = no + k % nv;
    const int sa = d.sp_a[sp], sb = d.sp_b[sp];
    const int la = d.sh_l[sa], lb = d.sh_l[sb];
    const double* A = d.atom_xyz + 3 * d.sh_atom[sa];
    const double* B = d.atom_xyz + 3 * d.sh_atom[sb];
    const double4_32a P = d.pp_P[L][g];
    double E[3][3][3][5];
    md_E1(la, lb, P.w, P.x - A[0], P.x - B[0], E[0]);
    md_E1(la, lb, P.w, P.y - A[1], P.y - B[1], E[1]);
    md_E1(la, lb, P.w, P.z - A[2], P.z - B[2], E[2]);
    const double* Cx = C + d.frag_moff[x];
    const int ao0 = d.frag_ao0[x];
    double acc[nh(kMaxLPair)];
    for (int h = 0; h < nh(L); ++h) acc[h] = 0.0;
    for (int ia = 0; ia < ncart(la); ++ia) {
        int ax, ay, az;
        cart_of(la, ia, ax, ay, az);
        const int mu = d.sh_ao[sa] + ia;
        for (int ib = 0; ib < ncart(lb); ++ib) {
            int bx, by, bz;
            cart_of(lb, ib, bx, by, bz);
            const int nu = d.sh_ao[sb] + ib;
            // phi_i phi_a over the ordered AO pairs of this shell pair (both orders when the shells differ)
            double w = Cx[mu * n + i] * Cx[nu * n + a];
            if (sa != sb) w += Cx[nu * n + i] * Cx[mu * n + a];
            w *= d.ao_scale[ao0 + mu] * d.ao_scale[ao0 + nu];
            for (int t = 0; t <= ax + bx; ++t)
                for (int u = 0; u <= ay + by; ++u)
                    for (int v = 0; v <= az + bz; ++v)
                        acc[hidx(t, u, v)] += w * E[0][ax][bx][t] * E[1][ay][by][u] * E[2][az][bz][v];
        }
    }
    const double sc = d.pp_K[L][g] * kSqrt2Pi52 / P.w * d.pp_rp[L][g];
    const int64_t row0 = uoff[x] + (int64_t)(hoff[x * kClasses + L] + (g - d.frag_pp0[x * kClasses + L]) * nh(L)) * nov;
    for (int h = 0; h < nh(L); ++h) U[row0 + (int64_t)h * nov + k] = acc[h] * sc;
}

// Below the Boys asymptotic switch: the unit-normalised base r F_n(T) (-2 alpha)^n / ((sqrt(pi)/2) p^{-1/2}
// q^{-1/2}) (as in the FP64 J-engine), out of line.
template <int L>
struct Ed2Base {
    double v[L + 1];
};
template <int L>
__device__ __noinline__ Ed2Base<L> ed2_table_base(const double* __restrict__ boys, double p, double q, double rp,
                                                  double rq, double R2, float Tf)
{
    Ed2Base<L> b;
    const double r = rsqrt(p + q);
    const double alpha = p * q * (r * r);
    double F[L + 1];
    boys_fp64<L>(boys, alpha * R2, boys_row(Tf), F);
    double pre = r * ((1.0 / kSqrtPiHalf) * (p * rp)) * (q * rq);
    const double m2a = -2.0 * alpha;
#pragma unroll
    for (int n2 = 0; n2 <= L; ++n2) {
        b.v[n2] = pre * F[n2];
        pre *= m2a;
    }
    return b;
}

struct Ed2Args {
    const double* U;       // transition Hermite densities (k_ed2_transition)
    const float2* Udf;     // the same as float-float pairs (the pair kernel's ket weights)
    const int64_t* uoff;   // [n_frag]
    const int* hoff;       // [n_frag * 5]
    const int* n_ov;       // [n_frag]
    const int* pair_of;    // chunk-local pair -> global pair
    const int64_t* goff;   // [2 * chunk pairs]: G offsets of (pair, side)
    double* G;
    float tau;
};

// Kets of class LK of fragment ky against the lane's bra pair (class LB): G[h][jj] += ...
// The contraction runs in float-float on the FP32 pipes: each R value (FP64) is split once per
// quartet, the weights are stored split, and G accumulates compensated unnormalised sums
// (ffa::acc_prod), ~2^-48 relative per term: the same accuracy class as FP64 for these sums of
// ~1e5 terms, at about a fifth of the FP64-pipe time of a DFMA per term on this part.
template <int LB, int LK>
__device__ __forceinline__ void ed2_kets(const Dev& d, const Ed2Args& a, int ky, int jb0, int nj, bool valid,
                                         const double4_32a& Pd, const float4& Pf, double rpP, float qP,
                                         ffa::dfacc (&G)[nh(LB)][ed2_cols(LB)])
{
    constexpr int NP = nh(LB), NQ = nh(LK), L = LB + LK, NR = nh(L), JC = ed2_cols(LB);
    const int k0 = d.frag_pp0[ky * kClasses + LK], k1 = k0 + d.frag_npp[ky * kClasses + LK];
    if (k0 >= k1) return;
    const int nov = a.n_ov[ky];
    const float2* __restrict__ Uk =
        a.Udf + a.uoff[ky] + (int64_t)a.hoff[ky * kClasses + LK] * nov + jb0;
    for (int k = k0; k < k1; ++k) {
        const float qQ = __ldg(d.pp_Q[LK] + k);
        const bool keep = valid && qP * qQ >= a.tau;
        if (!__any_sync(0xffffffffu, keep)) continue;
        const double4_32a Qd = d.pp_P[LK][k];
        const float4 Qf = __ldg(d.pp_Pf[LK] + k);
        const double X = Pd.x - Qd.x, Y = Pd.y - Qd.y, Z = Pd.z - Qd.z;
        const double R2 = fma(X, X, fma(Y, Y, Z * Z));
        const float Xf = Pf.x - Qf.x, Yf = Pf.y - Qf.y, Zf = Pf.z - Qf.z;
        const float R2f = fmaf(Xf, Xf, fmaf(Yf, Yf, Zf * Zf));
        const float pqf = Pf.w * Qf.w, sf = Pf.w + Qf.w;
        const bool asym = pqf * R2f >= (float)kBoysTmax * sf;
        const double yv = rsqrt_from_seed(R2, rsqrt_approx(R2f));
        double base[L + 1];
        base[0] = keep ? yv : 0.0;
        if constexpr (L > 0) {
            const double ny2 = -(yv * yv);
            static_for<L>([&](auto N) {
                constexpr int n2 = decltype(N)::value;
                if constexpr (n2 == 0)
                    base[1] = base[0] * ny2;
                else
                    base[n2 + 1] = base[n2] * (double(2 * n2 + 1) * ny2);
            });
        }
        if (!__all_sync(0xffffffffu, asym)) {
            if (!asym) {
                const Ed2Base<L> t = ed2_table_base<L>(d.boys, Pd.w, Qd.w, rpP, __ldg(d.pp_rp[LK] + k), R2,
                                                       __fdividef(pqf, sf) * R2f);
#pragma unroll
                for (int n2 = 0; n2 <= L; ++n2) base[n2] = keep ? t.v[n2] : 0.0;
            }
        }
        double R[NR];
        md_R<L, double>(R, base, X, Y, Z);
        ffa::df64 Rf[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) Rf[r] = ffa::from_double(R[r]);
        const float2* __restrict__ uq = Uk + (int64_t)(k - k0) * NQ * nov;
        static_for<NQ>([&](auto Jc) {
            constexpr TUV b = htuv(decltype(Jc)::value);
            constexpr bool odd = ((b.t + b.u + b.v) & 1) != 0;
            const float2* __restrict__ row = uq + (int64_t)decltype(Jc)::value * nov;
#pragma unroll
            for (int jj = 0; jj < JC; ++jj) {
                const float2 w2 = jj < nj ? __ldg(row + jj) : make_float2(0.0f, 0.0f);
                const ffa::df64 w(odd ? -w2.x : w2.x, odd ? -w2.y : w2.y);
                static_for<NP>([&](auto I) {
                    constexpr TUV c = htuv(decltype(I)::value);
                    ffa::acc_prod(G[decltype(I)::value][jj], Rf[hidx(c.t + b.t, c.u + b.u, c.v + b.v)], w);
                });
            }
        });
    }
}

// One warp per item (chunk-local pair q, side, first bra position, first jb column): item.x = 2 q + side
// (side 0: bra = x = pair_x, kets of y in classes >= LB; side 1: bra = y, kets of x in classes > LB),
// item.y = first bra primitive pair (global class-LB index), item.z = first jb column.
template <int LB>
__global__ void __launch_bounds__(128) k_ed2_pair(Dev d, Ed2Args a, const int4* __restrict__ items, int n_items)
{
    constexpr int NP = nh(LB), JC = ed2_cols(LB);
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (warp >= n_items) return;
    const int lane = threadIdx.x & 31;
    const int4 it = items[warp];
    const int q = it.x >> 1, side = it.x & 1;
    const int pr = a.pair_of[q];
    const int bx = side ? d.pair_y[pr] : d.pair_x[pr];
    const int ky = side ? d.pair_x[pr] : d.pair_y[pr];
    const int nov_k = a.n_ov[ky];
    const int jb0 = it.z, nj = min(JC, nov_k - jb0);
    const int bra_end = d.frag_pp0[bx * kClasses + LB] + d.frag_npp[bx * kClasses + LB];
    const int Pg = it.y + lane;
    const bool valid = Pg < bra_end;
    const int Pl = valid ? Pg : it.y;
    const double4_32a Pd = d.pp_P[LB][Pl];
    const float4 Pf = d.pp_Pf[LB][Pl];
    const double rpP = d.pp_rp[LB][Pl];
    const float qP = d.pp_Q[LB][Pl];
    ffa::dfacc G[NP][JC];
#pragma unroll
    for (int i = 0; i < NP; ++i)
#pragma unroll
        for (int j = 0; j < JC; ++j) G[i][j] = ffa::dfacc{0.0f, 0.0f};
    // ket classes: >= LB when x is the bra, > LB when y is (each class pair once)
    if (side == 0 && LB <= 0) ed2_kets<LB, 0>(d, a, ky, jb0, nj, valid, Pd, Pf, rpP, qP, G);
    if ((side == 0 && LB <= 1) || (side == 1 && LB < 1)) ed2_kets<LB, 1>(d, a, ky, jb0, nj, valid, Pd, Pf, rpP, qP, G);
    if ((side == 0 && LB <= 2) || (side == 1 && LB < 2)) ed2_kets<LB, 2>(d, a, ky, jb0, nj, valid, Pd, Pf, rpP, qP, G);
    if (!valid) return;
    // G rows of this bra pair: [(hoff + local pp * NP + h) * nov_k + jb]
    const int64_t row0 = a.goff[2 * q + side] +
                         (int64_t)(a.hoff[bx * kClasses + LB] + (Pg - d.frag_pp0[bx * kClasses + LB]) * NP) * nov_k + jb0;
#pragma unroll
    for (int i = 0; i < NP; ++i)
#pragma unroll
        for (int j = 0; j < JC; ++j)
            if (j < nj) a.G[row0 + (int64_t)i * nov_k + j] = (double)G[i][j].s + (double)G[i][j].c;
}

// Float-float copy of the transition densities (the pair kernel's ket weights).
__global__ void k_ed2_split(const double* __restrict__ U, float2* __restrict__ Udf, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const ffa::df64 v = ffa::from_double(U[i]);
        Udf[i] = make_float2(v.hi, v.lo);
    }
}

// E_D2 of each pair of the chunk: (ia|jb) = (sqrt(pi)/2) (sum_r U_x[r][ia] G_x[r][jb] + sum_r U_y[r][jb] G_y[r][ia]),
// rows r over the fragments' Hermite components; block (q, slice) takes the entries
// [slice * kEd2Entries, (slice + 1) * kEd2Entries) of pair q and writes its share to
// E_out[q * gridDim.y + slice] (the host adds the slices in order, so the sum is reproducible).
constexpr int kEd2Entries = 2048;

__global__ void __launch_bounds__(256) k_ed2_energy(Dev d, Ed2Args a, const double* __restrict__ C,
                                                    const double* __restrict__ eps, const int* __restrict__ nmo,
                                                    const int* __restrict__ n_herm, double* __restrict__ E_out)
{
    const int q = blockIdx.x;
    const int pr = a.pair_of[q];
    const int x = d.pair_x[pr], y = d.pair_y[pr];
    const int ox = d.frag_nocc[x], oy = d.frag_nocc[y];
    const int vx = nmo[x] - ox, vy = nmo[y] - oy;
    const int nvx = a.n_ov[x], nvy = a.n_ov[y];
    const int hx = n_herm[x], hy = n_herm[y];
    const double* __restrict__ Ux = a.U + a.uoff[x];
    const double* __restrict__ Uy = a.U + a.uoff[y];
    const double* __restrict__ Gx = a.G + a.goff[2 * q];      // [hx][nvy]
    const double* __restrict__ Gy = a.G + a.goff[2 * q + 1];  // [hy][nvx]
    const double* ex = eps + d.frag_ao0[x];
    const double* ey = eps + d.frag_ao0[y];
    double part = 0.0;
    const int e0 = blockIdx.y * kEd2Entries, e1 = min(nvx * nvy, e0 + kEd2Entries);
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const int ia = e / nvy, jb = e % nvy;
        double v = 0.0;
        for (int r = 0; r < hx; ++r) v = fma(Ux[(int64_t)r * nvx + ia], Gx[(int64_t)r * nvy + jb], v);
        for (int r = 0; r < hy; ++r) v = fma(Uy[(int64_t)r * nvy + jb], Gy[(int64_t)r * nvx + ia], v);
        v *= kSqrtPiHalf;
        const int i = ia / vx, aa = ia % vx, j = jb / vy, b = jb % vy;
        part += v * v / (ex[i] + ey[j] - ex[ox + aa] - ey[oy + b]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        E_out[(int64_t)q * gridDim.y + blockIdx.y] = 4.0 * s;
    }
}

}  // namespace

cudaError_t launch_ed2_transition(const Dev& d, const double* C, const int* nmo, const int64_t* uoff, const int* hoff,
                                  const int* n_ov, int max_ov, double* U, cudaStream_t s)
{
    for (int L = 0; L <= 2; ++L) {
        const int64_t n = (int64_t)d.n_pp[L] * max_ov;
        if (n == 0) continue;
        k_ed2_transition<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(d, L, C, nmo, uoff, hoff, n_ov, max_ov, U);
        note_launches(1);
    }
    return cudaGetLastError();
}

cudaError_t launch_ed2_split(const double* U, float2* Udf, int64_t n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_ed2_split<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(U, Udf, n);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_ed2_pairs(const Dev& d, const double* U, const float2* Udf, const int64_t* uoff, const int* hoff,
                             const int* n_ov, const int* pair_of, const int64_t* goff, double* G, double tau,
                             const int4* const items[3], const int n_items[3], cudaStream_t s)
{
    const Ed2Args a{U, Udf, uoff, hoff, n_ov, pair_of, goff, G, (float)tau};
    const int wpb = 4;
    if (n_items[0] > 0) k_ed2_pair<0><<<(n_items[0] + wpb - 1) / wpb, 32 * wpb, 0, s>>>(d, a, items[0], n_items[0]);
    if (n_items[1] > 0) k_ed2_pair<1><<<(n_items[1] + wpb - 1) / wpb, 32 * wpb, 0, s>>>(d, a, items[1], n_items[1]);
    if (n_items[2] > 0) k_ed2_pair<2><<<(n_items[2] + wpb - 1) / wpb, 32 * wpb, 0, s>>>(d, a, items[2], n_items[2]);
    note_launches((n_items[0] > 0) + (n_items[1] > 0) + (n_items[2] > 0));
    return cudaGetLastError();
}

cudaError_t launch_ed2_energy(const Dev& d, int n_pairs, int max_entries, const double* U, const int64_t* uoff,
                              const int* hoff, const int* n_ov, const int* pair_of, const int64_t* goff, const double* G,
                              const double* C, const double* eps, const int* nmo, const int* n_herm, double* E,
                              cudaStream_t s)
{
    if (n_pairs <= 0) return cudaSuccess;
    const Ed2Args a{U, nullptr, uoff, hoff, n_ov, pair_of, goff, const_cast<double*>(G), 0.0f};
    const dim3 grid(n_pairs, ed2_energy_slices(max_entries));
    k_ed2_energy<<<grid, 256, 0, s>>>(d, a, C, eps, nmo, n_herm, E);
    note_launches(1);
    return cudaGetLastError();
}

int ed2_cols_per_item(int LB) { return ed2_cols(LB); }

int ed2_energy_slices(int max_entries) { return std::max(1, (max_entries + kEd2Entries - 1) / kEd2Entries); }

}  // namespace fef
