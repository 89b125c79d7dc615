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
#include "common.cuh"
#include "internal.hpp"

namespace fef {

// ------------------------------------------------------------------------------------------ densities
__device__ inline int frag_of_shellpair(const Dev& d, int s)
{
    int lo = 0, hi = d.n_frag - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (d.frag_sp0[mid] <= s) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void k_hermite_density(Dev d, int L, const double* __restrict__ D)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    int npp = d.n_pp[L];
    if (g >= npp) return;
    int sp = d.pp_sp[L][g], ij = d.pp_ij[L][g];
    int sa = d.sp_a[sp], sb = d.sp_b[sp];
    int x = frag_of_shellpair(d, sp);
    int la = d.sh_l[sa], lb = d.sh_l[sb];
    const double* A = d.atom_xyz + 3 * d.sh_atom[sa];
    const double* B = d.atom_xyz + 3 * d.sh_atom[sb];
    double4_32a P = d.pp_P[L][g];
    double p = P.w;
    double E[3][3][3][5];
    md_E1(la, lb, p, P.x - A[0], P.x - B[0], E[0]);
    md_E1(la, lb, p, P.y - A[1], P.y - B[1], E[1]);
    md_E1(la, lb, p, P.z - A[2], P.z - B[2], E[2]);
    const int n = d.frag_nao[x];
    const double* Dx = D + d.frag_moff[x];
    const int ao0 = d.frag_ao0[x];
    double w = (sa == sb) ? 1.0 : 2.0;
    double acc[nh(kMaxLPair)];
    for (int k = 0; k < nh(L); ++k) acc[k] = 0.0;
    for (int ia = 0; ia < ncart(la); ++ia) {
        int ax, ay, az;
        cart_of(la, ia, ax, ay, az);
        int mu = d.sh_ao[sa] + ia;
        for (int ib = 0; ib < ncart(lb); ++ib) {
            int bx, by, bz;
            cart_of(lb, ib, bx, by, bz);
            int nu = d.sh_ao[sb] + ib;
            double dmn = w * Dx[mu * n + nu] * d.ao_scale[ao0 + mu] * d.ao_scale[ao0 + nu];
            for (int t = 0; t <= ax + bx; ++t)
                for (int u = 0; u <= ay + by; ++u)
                    for (int v = 0; v <= az + bz; ++v)
                        acc[hidx(t, u, v)] += dmn * E[0][ax][bx][t] * E[1][ay][by][u] * E[2][az][bz][v];
        }
    }
    double sc = d.pp_K[L][g] * kSqrt2Pi52 / p;
    for (int k = 0; k < nh(L); ++k) d.pp_Dh[L][(size_t)k * npp + g] = acc[k] * sc;
}

cudaError_t launch_hermite_density(const Dev& d, const double* D, cudaStream_t s)
{
    for (int L = 0; L < kClasses; ++L)
        if (d.n_pp[L] > 0) {
            k_hermite_density<<<(d.n_pp[L] + 127) / 128, 128, 0, s>>>(d, L, D);
            note_launches(1);
        }
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------ J-engine
// One warp per tile = (fragment pair x<y, up to 32 bra primitive pairs of class LP in x) against all
// ket primitive pairs of class LQ in y.  Lane i owns bra pair P_i: its centre, Hermite density and
// Hermite field accumulator stay in registers.  Ket data are warp-uniform loads.  The field on the
// ket pair is reduced across the warp with shuffles and added to global memory by lane 0.
// Shell quartets with Q_ab Q_cd < tau contribute nothing (Schwarz screening at shell level).
template <int LP, int LQ>
__global__ void __launch_bounds__(128) k_jengine(Dev d, const int2* __restrict__ tiles, int n_tiles, float tau,
                                                  double* __restrict__ e_pair)
{
    constexpr int NP = nh(LP), NQ = nh(LQ), L = LP + LQ, NR = nh(LP + LQ);
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n_tiles) return;
    const int2 tl = tiles[warp];
    const int x = d.pair_x[tl.x], y = d.pair_y[tl.x];
    const int bra_end = d.frag_pp0[x * kClasses + LP] + d.frag_npp[x * kClasses + LP];
    const int Pg = tl.y + lane;
    const bool valid = Pg < bra_end;
    const int Pl = valid ? Pg : tl.y;
    const int nP = d.n_pp[LP], nQ = d.n_pp[LQ];
    const double4_32a Pd = d.pp_P[LP][Pl];
    const float4 Pf = d.pp_Pf[LP][Pl];
    const float qP = valid ? d.pp_Q[LP][Pl] : 0.0f;
    double DP[NP], JP[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        DP[i] = valid ? d.pp_Dh[LP][(size_t)i * nP + Pl] : 0.0;
        JP[i] = 0.0;
    }
    const int k0 = d.frag_pp0[y * kClasses + LQ];
    const int k1 = k0 + d.frag_npp[y * kClasses + LQ];
    const double4_32a* __restrict__ QP = d.pp_P[LQ];
    const float4* __restrict__ QPf = d.pp_Pf[LQ];
    const float* __restrict__ QQ = d.pp_Q[LQ];
    const double* __restrict__ QD = d.pp_Dh[LQ];
    double* __restrict__ QJ = d.pp_Jh[LQ];
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
        const double r = rsqrt(Pd.w + Qd.w);
        const double alpha = Pd.w * Qd.w * (r * r);
        const double T = alpha * R2;
        const float Xf = Pf.x - Qf.x, Yf = Pf.y - Qf.y, Zf = Pf.z - Qf.z;
        const float Tf = __fdividef(Pf.w * Qf.w, Pf.w + Qf.w) * fmaf(Xf, Xf, fmaf(Yf, Yf, Zf * Zf));
        double F[L + 1];
        boys_fp64<L>(d.boys, T, boys_row(Tf), F);
        double base[L + 1];
        double pre = keep ? r : 0.0;
        const double m2a = -2.0 * alpha;
#pragma unroll
        for (int n = 0; n <= L; ++n) {
            base[n] = pre * F[n];
            pre *= m2a;
        }
        double R[NR];
        md_R<L, double>(R, base, X, Y, Z);
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            const TUV a = htuv(i);
            double acc = JP[i];
#pragma unroll
            for (int j = 0; j < NQ; ++j) {
                const TUV b = htuv(j);
                const double rr = R[hidx(a.t + b.t, a.u + b.u, a.v + b.v)];
                acc = ((b.t + b.u + b.v) & 1) ? fma(-rr, DQ[j], acc) : fma(rr, DQ[j], acc);
            }
            JP[i] = acc;
        }
#pragma unroll
        for (int j = 0; j < NQ; ++j) {
            const TUV b = htuv(j);
            double s = 0.0;
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                const TUV a = htuv(i);
                s = fma(R[hidx(a.t + b.t, a.u + b.u, a.v + b.v)], DP[i], s);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) atomicAdd(QJ + (size_t)j * nQ + k, ((b.t + b.u + b.v) & 1) ? -s : s);
        }
    }
    double e = 0.0;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        if (valid) atomicAdd(d.pp_Jh[LP] + (size_t)i * nP + Pg, JP[i]);
        e = fma(DP[i], JP[i], e);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if (lane == 0) atomicAdd(e_pair + tl.x, e);
}

template <int LP, int LQ>
static void launch_one(const Dev& d, const int2* t, int n, float tau, double* e, cudaStream_t s)
{
    if (n <= 0) return;
    const int warps_per_block = 4;
    k_jengine<LP, LQ><<<(n + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, s>>>(d, t, n, tau, e);
    note_launches(1);
}

cudaError_t launch_jengine(const Dev& d, const int2* tiles[kClasses][kClasses], const int* n_tiles, double tau,
                           double* e_pair, int /*mixed*/, cudaStream_t s)
{
    const float ft = (float)tau;
#define FEF_J(LP, LQ) launch_one<LP, LQ>(d, tiles[LP][LQ], n_tiles[LP * kClasses + LQ], ft, e_pair, s)
    FEF_J(0, 0); FEF_J(0, 1); FEF_J(0, 2); FEF_J(1, 0); FEF_J(1, 1); FEF_J(1, 2); FEF_J(2, 0); FEF_J(2, 1);
    FEF_J(2, 2);
#undef FEF_J
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------ back-transform
// J^x_{mu nu} = (c/p) sum_{P in shell pair of (mu, nu)} sum_tuv E^{mu nu}_tuv(P) Jh_P[tuv], scaled to
// normalised AOs.  One thread per (x, mu, nu).
__global__ void k_back_transform(Dev d, double* J)
{
    int x = blockIdx.y;
    int n = d.frag_nao[x];
    int nsh = d.frag_nsh[x], sh0 = d.frag_sh0[x], ao0 = d.frag_ao0[x];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
        int mu = e / n, nu = e % n;
        int s1 = d.ao_sh[ao0 + mu], s2 = d.ao_sh[ao0 + nu];
        int k1 = d.ao_k[ao0 + mu], k2 = d.ao_k[ao0 + nu];
        if (s1 > s2) {
            int t = s1; s1 = s2; s2 = t;
            t = k1; k1 = k2; k2 = t;
        }
        int a = s1 - sh0, b = s2 - sh0;
        int sp = d.frag_sp0[x] + a * (2 * nsh - a + 1) / 2 + (b - a);
        int L = d.sp_L[sp];
        int la = d.sh_l[s1], lb = d.sh_l[s2];
        int c1[3], c2[3];
        cart_of(la, k1, c1[0], c1[1], c1[2]);
        cart_of(lb, k2, c2[0], c2[1], c2[2]);
        const double* A = d.atom_xyz + 3 * d.sh_atom[s1];
        const double* B = d.atom_xyz + 3 * d.sh_atom[s2];
        int npp = d.n_pp[L];
        int np = d.sh_np[s1] * d.sh_np[s2];
        double acc = 0.0;
        for (int k = 0; k < np; ++k) {
            int g = d.sp_pp0[sp] + k;
            double4_32a P = d.pp_P[L][g];
            double E[3][3][3][5];
            md_E1(la, lb, P.w, P.x - A[0], P.x - B[0], E[0]);
            md_E1(la, lb, P.w, P.y - A[1], P.y - B[1], E[1]);
            md_E1(la, lb, P.w, P.z - A[2], P.z - B[2], E[2]);
            double v = 0.0;
            for (int t = 0; t <= c1[0] + c2[0]; ++t)
                for (int u = 0; u <= c1[1] + c2[1]; ++u)
                    for (int w = 0; w <= c1[2] + c2[2]; ++w)
                        v += E[0][c1[0]][c2[0]][t] * E[1][c1[1]][c2[1]][u] * E[2][c1[2]][c2[2]][w] *
                             d.pp_Jh[L][(size_t)hidx(t, u, w) * npp + g];
            acc += v * d.pp_K[L][g] * kSqrt2Pi52 / P.w;
        }
        J[d.frag_moff[x] + e] = acc * d.ao_scale[ao0 + mu] * d.ao_scale[ao0 + nu];
    }
}

cudaError_t launch_back_transform(const Dev& d, double* J, cudaStream_t s)
{
    dim3 g((d.max_nao * d.max_nao + 127) / 128, d.n_frag);
    k_back_transform<<<g, 128, 0, s>>>(d, J);
    note_launches(1);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------ Fock
// F^x = h^x + G[D^x] + V_env^x + J_env^x with G = C D (C: packed transposed Coulomb-minus-half-
// exchange tensor, see setup.cu), plus E_int[x] = tr[D (h + G/2)] + E_nn(x) and tr[D omega]
// (omega = V_env + J_env).  One block per fragment; thread per packed row pq = (mu <= nu).
__global__ void k_fock_assemble(Dev d, const double* h, const double* Venv, const double* Jenv, const double* eric,
                                const double* D, double* F, double* omega, const double* e_nn, double* E_int,
                                double* tr_omega)
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
    double eint = 0.0, eom = 0.0;
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
        double om = (Venv ? Venv[o] : 0.0) + (Jenv ? Jenv[o] : 0.0);
        eint += w * Dx[mu * n + nu] * (h[o] + 0.5 * g);
        eom += w * Dx[mu * n + nu] * om;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        eint += __shfl_xor_sync(0xffffffffu, eint, o);
        eom += __shfl_xor_sync(0xffffffffu, eom, o);
    }
    __shared__ double r1[32], r2[32];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (lane == 0) {
        r1[warp] = eint;
        r2[warp] = eom;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < nw; ++w) {
            a += r1[w];
            b += r2[w];
        }
        if (E_int) E_int[x] = a + e_nn[x];
        if (tr_omega) tr_omega[x] = b;
    }
}

cudaError_t launch_fock_energy(const Dev& d, const double* h, const double* Venv, const double* Jenv,
                               const double* eric, const double* D, double* F, double* omega, const double* e_nn,
                               double* E_int, double* tr_omega, cudaStream_t s)
{
    size_t smem = sizeof(double) * (size_t)d.max_nao * (d.max_nao + 1) / 2;
    k_fock_assemble<<<d.n_frag, 256, smem, s>>>(d, h, Venv, Jenv, eric, D, F, omega, e_nn, E_int, tr_omega);
    note_launches(1);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------ energies
// E_xy = tr[D^x V^y] + tr[D^y V^x] + tr[D^x J[D^y]] + E_nn(x,y) per pair; E_frag[x] = E_int[x] +
// (1/2) sum_{y in N(x)} E_xy; E_total = sum_x E_int + sum_pairs E_xy (one block, fixed order).
__global__ void k_pair_energy(Dev d, const double* e_J, const double* tr_xy, const double* tr_yx, const double* e_nn,
                              double* E_pair)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < d.n_pairs) E_pair[p] = tr_xy[p] + tr_yx[p] + e_J[p] + e_nn[p];
}

__global__ void k_frag_energy(Dev d, const double* E_int, const double* E_pair, double* E_frag)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= d.n_frag) return;
    double e = 0.0;
    for (int c = d.frag_nbr0[x]; c < d.frag_nbr0[x + 1]; ++c) e += E_pair[d.nbr_pair[c]];
    E_frag[x] = E_int[x] + 0.5 * e;
}

__global__ void k_total_energy(Dev d, const double* E_int, const double* E_pair, double* E_tot)
{
    __shared__ double red[256];
    double a = 0.0;
    for (int i = threadIdx.x; i < d.n_frag; i += blockDim.x) a += E_int[i];
    for (int i = threadIdx.x; i < d.n_pairs; i += blockDim.x) a += E_pair[i];
    red[threadIdx.x] = a;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *E_tot = red[0];
}

cudaError_t launch_energies(const Dev& d, const double* e_J, const double* tr_xy, const double* tr_yx,
                            const double* e_nn_pair, const double* E_int, double* E_pair, double* E_frag,
                            double* E_tot, cudaStream_t s)
{
    if (d.n_pairs > 0) {
        k_pair_energy<<<(d.n_pairs + 255) / 256, 256, 0, s>>>(d, e_J, tr_xy, tr_yx, e_nn_pair, E_pair);
        note_launches(1);
    }
    k_frag_energy<<<(d.n_frag + 255) / 256, 256, 0, s>>>(d, E_int, E_pair, E_frag);
    note_launches(1);
    k_total_energy<<<1, 256, 0, s>>>(d, E_int, E_pair, E_tot);
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
