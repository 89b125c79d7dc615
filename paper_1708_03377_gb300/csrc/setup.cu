// Geometry-time kernels of the FEF context: basis normalisation, the Boys table, primitive pairs,
// one-electron matrices (S, h = T + V_own), the intra-fragment two-electron tensor and its
// Coulomb-minus-half-exchange form, Schwarz factors, the fragment neighbour test, the environment
// nuclear attraction h~ (paper, "Fragment Mean Field", the equation after Eq. wc) and nuclear
// repulsion.  All integrals use McMurchie-Davidson Hermite expansions (common.cuh).
#include <algorithm>

#include "common.cuh"
#include "internal.hpp"

namespace fef {

// ------------------------------------------------------------------------------------------ prepare
__global__ void k_prepare(int n_atoms, const double* xyz_A, double* xyz_bohr, int n_prims, const double* exps,
                          const double* coef_raw, const int* p_l, double* coef)
{
    const double bohr_per_A = 1.0 / 0.529177210903;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 3 * n_atoms) xyz_bohr[i] = xyz_A[i] * bohr_per_A;
    if (i < n_prims) coef[i] = coef_raw[i] * prim_norm(exps[i], p_l[i]);
}

cudaError_t launch_prepare(const Dev& d, const double* xyz_A, double* atom_xyz, double* p_coef_out,
                           const double* p_coef_raw, const int* p_l, int n_prims, cudaStream_t s)
{
    int n = max(3 * d.n_atoms, n_prims);
    k_prepare<<<(n + 255) / 256, 256, 0, s>>>(d.n_atoms, xyz_A, atom_xyz, n_prims, d.p_exp, p_coef_raw, p_l,
                                              p_coef_out);
    note_launches(1);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------ Boys table
// F_n(T_k) for n = 0..14 by the series F_N(T) = exp(-T) sum_i (2T)^i / ((2N+1)(2N+3)...(2N+2i+1))
// (all terms positive, compensated summation) and downward recursion
// F_n = (2T F_{n+1} + exp(-T)) / (2n+1); stored as Taylor coefficients F_{m+j}(T_k)/j!.
__global__ void k_boys_table(double* table)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kBoysRows) return;
    const int N = kBoysM - 1 + kBoysOrder;  // 14
    const double T = k * kBoysH;
    double term = 1.0 / (2.0 * N + 1.0), sum = term, comp = 0.0;
    for (int i = 1; i < 4000; ++i) {
        term *= 2.0 * T / (2.0 * N + 2.0 * i + 1.0);
        double y = term - comp;
        double t = sum + y;
        comp = (t - sum) - y;
        sum = t;
        if (term < 1e-20 * sum) break;
    }
    const double e = exp(-T);
    double F[kBoysM + kBoysOrder];
    F[N] = e * sum;
    for (int n = N - 1; n >= 0; --n) F[n] = (2.0 * T * F[n + 1] + e) / (2.0 * n + 1.0);
    double* row = table + (size_t)k * kBoysRowLen;
    double fact = 1.0;
    for (int m = 0; m < kBoysM; ++m) {
        fact = 1.0;
        for (int j = 0; j <= kBoysOrder; ++j) {
            if (j > 0) fact *= j;
            row[m * kBoysBlock + j] = F[m + j] / fact;
        }
        row[m * kBoysBlock + kBoysOrder + 1] = (m == 0) ? T : 0.0;
    }
}

cudaError_t launch_boys_table(double* table, cudaStream_t s)
{
    k_boys_table<<<(kBoysRows + 127) / 128, 128, 0, s>>>(table);
    note_launches(1);
    return cudaGetLastError();
}

// FP32 table for the mixed-precision core, from the FP64 table: row k, block m holds F_{m+j}(T_k)/j!
// (j = 0..4); F_n for n <= 8 is block n coefficient 0, for n > 8 block 8 coefficient n-8 times (n-8)!.
__global__ void k_boys_table32(const double* t64, float* t32)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kBoys32Rows) return;
    const double* row = t64 + (size_t)k * kBoysRowLen;
    double F[kBoysM + kBoys32Order];
    for (int n = 0; n < kBoysM; ++n) F[n] = row[n * kBoysBlock];
    double fact = 1.0;
    for (int j = 1; j <= kBoys32Order; ++j) {
        fact *= j;
        F[kBoysM - 1 + j] = row[(kBoysM - 1) * kBoysBlock + j] * fact;
    }
    float* out = t32 + (size_t)k * kBoysRowLen;
    for (int m = 0; m < kBoysM; ++m) {
        double f = 1.0;
        for (int j = 0; j <= kBoys32Order; ++j) {
            if (j > 0) f *= j;
            out[m * kBoysBlock + j] = (float)(F[m + j] / f);
        }
        for (int j = kBoys32Order + 1; j < kBoysBlock; ++j) out[m * kBoysBlock + j] = 0.0f;
    }
    out[kBoys32Order + 3] = (float)row[kBoysOrder + 1];  // T_k
}

cudaError_t launch_boys_table32(const double* table64, float* table32, cudaStream_t s)
{
    k_boys_table32<<<(kBoys32Rows + 127) / 128, 128, 0, s>>>(table64, table32);
    note_launches(1);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------ AO scale
// Raw self-overlap of contracted AO (lx,ly,lz): sum_ij c_i c_j (pi/p)^{3/2} prod_d E^{l_d l_d}_0 with
// both primitives on one centre (X_PA = X_PB = 0); the AO scale makes it 1.
__global__ void k_ao_scale(Dev d, double* ao_scale, int n_ao_total)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_ao_total) return;
    int sh = d.ao_sh[g], k = d.ao_k[g];
    int l = d.sh_l[sh], np = d.sh_np[sh], p0 = d.sh_p0[sh];
    int lc[3];
    cart_of(l, k, lc[0], lc[1], lc[2]);
    double S = 0.0;
    for (int i = 0; i < np; ++i)
        for (int j = 0; j < np; ++j) {
            double a = d.p_exp[p0 + i], b = d.p_exp[p0 + j], p = a + b;
            double v = d.p_coef[p0 + i] * d.p_coef[p0 + j] * pow(kPi / p, 1.5);
            for (int dd = 0; dd < 3; ++dd) {
                double E[3][3][5];
                md_E1(lc[dd], lc[dd], p, 0.0, 0.0, E);
                v *= E[lc[dd]][lc[dd]][0];
            }
            S += v;
        }
    ao_scale[g] = 1.0 / sqrt(S);
}

cudaError_t launch_ao_scale(const Dev& d, double* ao_scale, int n_ao_total, const int*, cudaStream_t s)
{
    k_ao_scale<<<(n_ao_total + 127) / 128, 128, 0, s>>>(d, ao_scale, n_ao_total);
    note_launches(1);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------ prim pairs
// P = (a A + b B)/p, p = a + b, K = c_i c_j exp(-a b/p |AB|^2), for every primitive pair.
__global__ void k_prim_pairs(Dev d, int L, double4_32a* P, float4* Pf, double* K, float4* Pr, double* rp)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= d.n_pp[L]) return;
    int sp = d.pp_sp[L][g], ij = d.pp_ij[L][g];
    int sa = d.sp_a[sp], sb = d.sp_b[sp];
    int pa = d.sh_p0[sa] + (ij >> 4), pb = d.sh_p0[sb] + (ij & 15);
    const double* A = d.atom_xyz + 3 * d.sh_atom[sa];
    const double* B = d.atom_xyz + 3 * d.sh_atom[sb];
    double a = d.p_exp[pa], b = d.p_exp[pb], p = a + b;
    double R2 = 0.0, Pc[3];
    for (int k = 0; k < 3; ++k) {
        Pc[k] = (a * A[k] + b * B[k]) / p;
        R2 += (A[k] - B[k]) * (A[k] - B[k]);
    }
    P[g] = make_double4_32a(Pc[0], Pc[1], Pc[2], p);
    Pf[g] = make_float4((float)Pc[0], (float)Pc[1], (float)Pc[2], (float)p);
    const double* anc = d.atom_xyz + 3 * d.frag_atom0[frag_of_shellpair(d, sp)];
    Pr[g] = make_float4((float)(Pc[0] - anc[0]), (float)(Pc[1] - anc[1]), (float)(Pc[2] - anc[2]), (float)p);
    K[g] = d.p_coef[pa] * d.p_coef[pb] * exp(-a * b / p * R2);
    rp[g] = 1.0 / sqrt(p);
}

cudaError_t launch_prim_pairs(const Dev& d, double4_32a* P[kClasses], float4* Pf[kClasses], double* K[kClasses],
                              float4* Pr[kClasses], double* rp[kClasses], cudaStream_t s)
{
    for (int L = 0; L < kClasses; ++L)
        if (d.n_pp[L] > 0) {
            k_prim_pairs<<<(d.n_pp[L] + 127) / 128, 128, 0, s>>>(d, L, P[L], Pf[L], K[L], Pr[L], rp[L]);
            note_launches(1);
        }
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------ one-electron
struct AOPair {
    int la, lb;
    int ca[3], cb[3];
    int pa0, pb0, na, nb;
    const double* A;
    const double* B;
    double scale;
};

__device__ inline AOPair ao_pair(const Dev& d, int x, int mu, int nu)
{
    AOPair q;
    int gmu = d.frag_ao0[x] + mu, gnu = d.frag_ao0[x] + nu;
    int sa = d.ao_sh[gmu], sb = d.ao_sh[gnu];
    q.la = d.sh_l[sa];
    q.lb = d.sh_l[sb];
    cart_of(q.la, d.ao_k[gmu], q.ca[0], q.ca[1], q.ca[2]);
    cart_of(q.lb, d.ao_k[gnu], q.cb[0], q.cb[1], q.cb[2]);
    q.pa0 = d.sh_p0[sa];
    q.pb0 = d.sh_p0[sb];
    q.na = d.sh_np[sa];
    q.nb = d.sh_np[sb];
    q.A = d.atom_xyz + 3 * d.sh_atom[sa];
    q.B = d.atom_xyz + 3 * d.sh_atom[sb];
    q.scale = d.ao_scale[gmu] * d.ao_scale[gnu];
    return q;
}

// 1D overlap integrals E^{ij}_0 for j up to jmax <= 4 (kinetic needs j+2).
__device__ inline void e1_overlap(int imax, int jmax, double p, double XPA, double XPB, double (*E)[5][7])
{
    const double h = 0.5 / p;
    for (int i = 0; i <= imax; ++i)
        for (int j = 0; j <= jmax; ++j)
            for (int t = 0; t < 7; ++t) E[i][j][t] = 0.0;
    E[0][0][0] = 1.0;
    for (int i = 0; i < imax; ++i)
        for (int t = 0; t <= i + 1; ++t) {
            double v = XPA * (t <= i ? E[i][0][t] : 0.0);
            if (t > 0) v += h * E[i][0][t - 1];
            if (t + 1 <= i) v += (t + 1) * E[i][0][t + 1];
            E[i + 1][0][t] = v;
        }
    for (int i = 0; i <= imax; ++i)
        for (int j = 0; j < jmax; ++j)
            for (int t = 0; t <= i + j + 1 && t < 7; ++t) {
                double v = XPB * (t <= i + j ? E[i][j][t] : 0.0);
                if (t > 0) v += h * E[i][j][t - 1];
                if (t + 1 <= i + j) v += (t + 1) * E[i][j][t + 1];
                E[i][j + 1][t] = v;
            }
}

// Nuclear attraction of one primitive pair to a set of point charges:
//   sum_C -Z_C (2 pi/p) sum_tuv E^x_t E^y_u E^z_v R_tuv(p, P - C).
__device__ inline double nuclear_prim(const Dev& d, const AOPair& q, double a, double b, const double (*Ex)[3][5],
                                      const double (*Ey)[3][5], const double (*Ez)[3][5], const double* P, double p,
                                      int atom0, int natoms)
{
    int L = q.la + q.lb;
    double acc = 0.0;
    double R[nh(kMaxLPair)], base[kMaxLPair + 1], F[kMaxLPair + 1];
    for (int c = atom0; c < atom0 + natoms; ++c) {
        const double* C = d.atom_xyz + 3 * c;
        double X = P[0] - C[0], Y = P[1] - C[1], Z = P[2] - C[2];
        double T = p * (X * X + Y * Y + Z * Z);
        boys_fp64_rt(d.boys, T, L, F);
        double f = 1.0;
        for (int n = 0; n <= L; ++n) {
            base[n] = f * F[n];
            f *= -2.0 * p;
        }
        md_R_rt(L, R, base, X, Y, Z);
        double v = 0.0;
        for (int t = 0; t <= q.ca[0] + q.cb[0]; ++t)
            for (int u = 0; u <= q.ca[1] + q.cb[1]; ++u)
                for (int w = 0; w <= q.ca[2] + q.cb[2]; ++w)
                    v += Ex[q.ca[0]][q.cb[0]][t] * Ey[q.ca[1]][q.cb[1]][u] * Ez[q.ca[2]][q.cb[2]][w] * R[hidx(t, u, w)];
        acc -= d.atom_Z[c] * v;
    }
    return acc * 2.0 * kPi / p;
}

// S, T and V(own nuclei) for every (x, mu, nu); h = T + V.
__global__ void k_one_electron(Dev d, double* Sout, double* hout)
{
    int x = blockIdx.y;
    int n = d.frag_nao[x];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
        int mu = e / n, nu = e % n;
        AOPair q = ao_pair(d, x, mu, nu);
        double S = 0.0, T = 0.0, V = 0.0;
        for (int i = 0; i < q.na; ++i)
            for (int j = 0; j < q.nb; ++j) {
                double a = d.p_exp[q.pa0 + i], b = d.p_exp[q.pb0 + j], p = a + b;
                double cc = d.p_coef[q.pa0 + i] * d.p_coef[q.pb0 + j];
                double P[3], R2 = 0.0;
                double Es[3][3][5][7];
                double E[3][3][3][5];
                for (int k = 0; k < 3; ++k) {
                    P[k] = (a * q.A[k] + b * q.B[k]) / p;
                    R2 += (q.A[k] - q.B[k]) * (q.A[k] - q.B[k]);
                    e1_overlap(q.ca[k], q.cb[k] + 2, p, P[k] - q.A[k], P[k] - q.B[k], Es[k]);
                    md_E1(q.la, q.lb, p, P[k] - q.A[k], P[k] - q.B[k], E[k]);
                }
                double K = cc * exp(-a * b / p * R2);
                double s1[3], t1[3];
                for (int k = 0; k < 3; ++k) {
                    int i1 = q.ca[k], j1 = q.cb[k];
                    s1[k] = Es[k][i1][j1][0];
                    // d^2/dx^2 acting on x_B^j exp(-b x_B^2): j(j-1) x^{j-2} - 2b(2j+1) x^j + 4b^2 x^{j+2}
                    double v = -2.0 * b * (2 * j1 + 1) * Es[k][i1][j1][0] + 4.0 * b * b * Es[k][i1][j1 + 2][0];
                    if (j1 >= 2) v += j1 * (j1 - 1) * Es[k][i1][j1 - 2][0];
                    t1[k] = v;
                }
                double pre = K * pow(kPi / p, 1.5);
                S += pre * s1[0] * s1[1] * s1[2];
                T += pre * -0.5 * (t1[0] * s1[1] * s1[2] + s1[0] * t1[1] * s1[2] + s1[0] * s1[1] * t1[2]);
                V += K * nuclear_prim(d, q, a, b, E[0], E[1], E[2], P, p, d.frag_atom0[x], d.frag_nat[x]);
            }
        int64_t o = d.frag_moff[x] + e;
        Sout[o] = S * q.scale;
        hout[o] = (T + V) * q.scale;
    }
}

cudaError_t launch_one_electron(const Dev& d, double* S, double* h, cudaStream_t s)
{
    dim3 g((d.max_nao * d.max_nao + 127) / 128, d.n_frag);
    k_one_electron<<<g, 128, 0, s>>>(d, S, h);
    note_launches(1);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------ far field
// Fragment pairs beyond the cutoff interact through the multipoles of each fragment's nuclei and
// electrons about its nuclear-charge centroid c_x (charge, dipole, second moments), the potential of
// y Taylor-expanded to second order about c_x (the far-field extension of Eq. wc's sum over y).
// Moment integrals (geometry time): M[k][mu][nu] = <mu|(r - c_x)^k|nu>, k = 1, x, y, z, xx, xy, xz,
// yy, yz, zz, at 10 frag_moff[x] + k n^2, from the Hermite expansion of each primitive product:
// int (x - c)^m Lambda_t dx = sqrt(pi/p) H^m_t with H^0_0 = 1, H^1_0 = X_PC, H^1_1 = 1,
// H^2_0 = X_PC^2 + 1/(2p), H^2_1 = 2 X_PC, H^2_2 = 2.
__global__ void k_moment_integrals(Dev d, const double* __restrict__ cen, double* M)
{
    const int x = blockIdx.y;
    const int n = d.frag_nao[x];
    const double* c = cen + 3 * x;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
        const int mu = e / n, nu = e % n;
        AOPair q = ao_pair(d, x, mu, nu);
        double acc[10] = {};
        for (int i = 0; i < q.na; ++i)
            for (int j = 0; j < q.nb; ++j) {
                const double a = d.p_exp[q.pa0 + i], b = d.p_exp[q.pb0 + j], p = a + b;
                const double cc = d.p_coef[q.pa0 + i] * d.p_coef[q.pb0 + j];
                double P[3], R2 = 0.0, m[3][3];
                double E[3][3][3][5];
                for (int k = 0; k < 3; ++k) {
                    P[k] = (a * q.A[k] + b * q.B[k]) / p;
                    R2 += (q.A[k] - q.B[k]) * (q.A[k] - q.B[k]);
                    md_E1(q.la, q.lb, p, P[k] - q.A[k], P[k] - q.B[k], E[k]);
                    const double* Et = E[k][q.ca[k]][q.cb[k]];
                    const int tmax = q.ca[k] + q.cb[k];
                    const double X = P[k] - c[k];
                    const double e0 = Et[0], e1 = tmax >= 1 ? Et[1] : 0.0, e2 = tmax >= 2 ? Et[2] : 0.0;
                    m[k][0] = e0;
                    m[k][1] = X * e0 + e1;
                    m[k][2] = (X * X + 0.5 / p) * e0 + 2.0 * X * e1 + 2.0 * e2;
                }
                const double pre = cc * exp(-a * b / p * R2) * pow(kPi / p, 1.5);
                const int kk[10][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0},
                                       {1, 1, 0}, {1, 0, 1}, {0, 2, 0}, {0, 1, 1}, {0, 0, 2}};
                for (int k = 0; k < 10; ++k) acc[k] += pre * m[0][kk[k][0]] * m[1][kk[k][1]] * m[2][kk[k][2]];
            }
        for (int k = 0; k < 10; ++k) M[10 * d.frag_moff[x] + (int64_t)k * n * n + e] = acc[k] * q.scale;
    }
}

cudaError_t launch_moment_integrals(const Dev& d, const double* cen, double* M, cudaStream_t s)
{
    dim3 g((d.max_nao * d.max_nao + 127) / 128, d.n_frag);
    k_moment_integrals<<<g, 128, 0, s>>>(d, cen, M);
    note_launches(1);
    return cudaGetLastError();
}

// Multipoles of every fragment for the densities D: mult[x][k] = Mnuc[x][k] - tr(D^x M_k), one block
// per fragment (charge, dipole, second moments xx xy xz yy yz zz).
__global__ void k_far_multipoles(Dev d, const double* __restrict__ M, const double* __restrict__ Mnuc,
                                 const double* __restrict__ D, double* mult)
{
    const int x = blockIdx.x;
    const int n = d.frag_nao[x];
    const double* Dx = D + d.frag_moff[x];
    const double* Mx = M + 10 * d.frag_moff[x];
    __shared__ double red[10][8];
    double acc[10] = {};
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const double de = Dx[e];
        for (int k = 0; k < 10; ++k) acc[k] = fma(de, Mx[(int64_t)k * n * n + e], acc[k]);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = 0; k < 10; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[k][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < 10) {
        double t = 0.0;
        for (int j = 0; j < (int)(blockDim.x >> 5); ++j) t += red[threadIdx.x][j];
        mult[10 * x + threadIdx.x] = Mnuc[10 * x + threadIdx.x] - t;
    }
}

// Potential of y's multipoles (my: charge, dipole, second moments) at R = c_x - c_y, Taylor terms to
// second order: phi = q T - mu.T1 + (1/2) M2 : T2 with T_n the derivatives of 1/|R| in closed form,
// its gradient gy and Hessian Hy.
__device__ __forceinline__ void multipole_potential(const double R[3], const double* __restrict__ my, double& p,
                                                    double gy[3], double Hy[3][3])
{
    const double q = my[0];
    const double mu[3] = {my[1], my[2], my[3]};
    const double M2[3][3] = {{my[4], my[5], my[6]}, {my[5], my[7], my[8]}, {my[6], my[8], my[9]}};
    const double r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
    const double ir = rsqrt(r2), ir2 = ir * ir;
    const double ir3 = ir * ir2, ir5 = ir3 * ir2, ir7 = ir5 * ir2, ir9 = ir7 * ir2;
    double MR[3];
    for (int a = 0; a < 3; ++a) MR[a] = M2[a][0] * R[0] + M2[a][1] * R[1] + M2[a][2] * R[2];
    const double RMR = R[0] * MR[0] + R[1] * MR[1] + R[2] * MR[2];
    const double trM = M2[0][0] + M2[1][1] + M2[2][2];
    const double muR = mu[0] * R[0] + mu[1] * R[1] + mu[2] * R[2];
    // phi = q/r + mu.R/r^3 + (1/2)(3 RMR/r^5 - trM/r^3)
    p = q * ir + muR * ir3 + 0.5 * (3.0 * RMR * ir5 - trM * ir3);
    for (int c = 0; c < 3; ++c) {
        // g_c = q T_c - sum_a mu_a T_ac + (1/2) sum_ab M_ab T_abc
        const double Tc = -R[c] * ir3;
        const double muT2 = 3.0 * muR * R[c] * ir5 - mu[c] * ir3;
        const double MT3 = -15.0 * RMR * R[c] * ir7 + 3.0 * (2.0 * MR[c] + trM * R[c]) * ir5;
        gy[c] = q * Tc - muT2 + 0.5 * MT3;
        for (int e = 0; e < 3; ++e) {
            const double dce = c == e ? 1.0 : 0.0;
            const double T2 = (3.0 * R[c] * R[e] - r2 * dce) * ir5;
            const double muT3 = -15.0 * muR * R[c] * R[e] * ir7 + 3.0 * (mu[c] * R[e] + mu[e] * R[c] + muR * dce) * ir5;
            const double MT4 = 105.0 * RMR * R[c] * R[e] * ir9
                               - 15.0 * (RMR * dce + 2.0 * R[c] * MR[e] + 2.0 * R[e] * MR[c] + trM * R[c] * R[e]) * ir7
                               + 3.0 * (trM * dce + 2.0 * M2[c][e]) * ir5;
            Hy[c][e] = q * T2 - muT3 + 0.5 * MT4;
        }
    }
}

// Potential of the far fragments at c_x, summed: pot[x] = (phi, grad phi[3], hess phi[xx xy xz yy yz zz]),
// and E_far[x] = (1/2) sum_y (q_x phi + mu_x . g + (1/2) M2_x : H).  One thread per fragment; pairs
// within the cutoff (the neighbour list) are skipped.
__global__ void k_far_potential(Dev d, const double* __restrict__ cen, const double* __restrict__ mult, double* pot,
                                double* E_far)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= d.n_frag) return;
    double ph = 0.0, g[3] = {}, H[3][3] = {};
    double e_sum = 0.0;
    const double* cx = cen + 3 * x;
    const double* mx = mult + 10 * x;
    const double Mx[3][3] = {{mx[4], mx[5], mx[6]}, {mx[5], mx[7], mx[8]}, {mx[6], mx[8], mx[9]}};
    for (int y = 0; y < d.n_frag; ++y) {
        if (y == x) continue;
        bool near = false;
        for (int c = d.frag_nbr0[x]; c < d.frag_nbr0[x + 1]; ++c) near = near || d.nbr[c] == y;
        if (near) continue;
        double R[3];
        for (int a = 0; a < 3; ++a) R[a] = cx[a] - cen[3 * y + a];
        double p, gy[3], Hy[3][3];
        multipole_potential(R, mult + 10 * y, p, gy, Hy);
        double exy = mx[0] * p;
        for (int c = 0; c < 3; ++c) {
            exy += mx[1 + c] * gy[c];
            for (int e = 0; e < 3; ++e) exy += 0.5 * Mx[c][e] * Hy[c][e];
        }
        e_sum += exy;
        ph += p;
        for (int c = 0; c < 3; ++c) {
            g[c] += gy[c];
            for (int e = 0; e < 3; ++e) H[c][e] += Hy[c][e];
        }
    }
    double* o = pot + 10 * x;
    o[0] = ph;
    o[1] = g[0]; o[2] = g[1]; o[3] = g[2];
    o[4] = H[0][0]; o[5] = H[0][1]; o[6] = H[0][2]; o[7] = H[1][1]; o[8] = H[1][2]; o[9] = H[2][2];
    E_far[x] = 0.5 * e_sum;
}

// The same expansion over the neighbours within the cutoff instead (the learned start's multipole
// estimate of the environment operator; no energy).  One warp per fragment, lanes over neighbours.
__global__ void k_near_multipole_potential(Dev d, const double* __restrict__ cen, const double* __restrict__ mult,
                                           double* pot)
{
    const int x = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (x >= d.n_frag) return;
    double acc[10] = {};
    const double* cx = cen + 3 * x;
    for (int c = d.frag_nbr0[x] + lane; c < d.frag_nbr0[x + 1]; c += 32) {
        const int y = d.nbr[c];
        double R[3];
        for (int a = 0; a < 3; ++a) R[a] = cx[a] - cen[3 * y + a];
        double p, gy[3], Hy[3][3];
        multipole_potential(R, mult + 10 * y, p, gy, Hy);
        acc[0] += p;
        acc[1] += gy[0]; acc[2] += gy[1]; acc[3] += gy[2];
        acc[4] += Hy[0][0]; acc[5] += Hy[0][1]; acc[6] += Hy[0][2]; acc[7] += Hy[1][1]; acc[8] += Hy[1][2];
        acc[9] += Hy[2][2];
    }
    for (int k = 0; k < 10; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) pot[10 * x + k] = v;
    }
}

// F^x and omega_x += -(phi S + grad phi . <r> + (1/2) hess phi : <r r>) (the density derivative of
// the far-field energy; off-diagonal second moments count twice).
__global__ void k_far_fock(Dev d, const double* __restrict__ M, const double* __restrict__ pot, double* F,
                           double* omega)
{
    const int x = blockIdx.y;
    const int n = d.frag_nao[x];
    const double* Mx = M + 10 * d.frag_moff[x];
    const double* o = pot + 10 * x;
    const double w[10] = {o[0], o[1], o[2], o[3], 0.5 * o[4], o[5], o[6], 0.5 * o[7], o[8], 0.5 * o[9]};
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int k = 0; k < 10; ++k) v = fma(w[k], Mx[(int64_t)k * n * n + e], v);
        const int64_t i = d.frag_moff[x] + e;
        if (F) F[i] -= v;
        if (omega) omega[i] -= v;
    }
}

// E_frag[x] += E_far[x]; E_tot = sum_x E_frag[x] (one block).
__global__ void k_far_energy(Dev d, const double* __restrict__ E_far, double* E_frag, double* E_tot)
{
    __shared__ double red[256];
    double a = 0.0;
    for (int x = threadIdx.x; x < d.n_frag; x += blockDim.x) {
        const double e = E_frag[x] + E_far[x];
        E_frag[x] = e;
        a += e;
    }
    red[threadIdx.x] = a;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) *E_tot = red[0];
}

cudaError_t launch_far_field(const Dev& d, const double* M, const double* Mnuc, const double* cen, const double* D,
                             double* mult, double* pot, double* E_far, double* F, double* omega, cudaStream_t s)
{
    if (d.n_frag <= 1) return cudaSuccess;
    k_far_multipoles<<<d.n_frag, 128, 0, s>>>(d, M, Mnuc, D, mult);
    k_far_potential<<<(d.n_frag + 127) / 128, 128, 0, s>>>(d, cen, mult, pot, E_far);
    dim3 g((d.max_nao * d.max_nao + 127) / 128, d.n_frag);
    k_far_fock<<<g, 128, 0, s>>>(d, M, pot, F, omega);
    note_launches(3);
    return cudaGetLastError();
}

cudaError_t launch_near_multipole_field(const Dev& d, const double* M, const double* Mnuc, const double* cen,
                                       const double* D, double* mult, double* pot, double* omega, int64_t n_omega,
                                       cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(omega, 0, sizeof(double) * n_omega, s);
    if (e != cudaSuccess || d.n_frag <= 0) return e;
    k_far_multipoles<<<d.n_frag, 128, 0, s>>>(d, M, Mnuc, D, mult);
    k_near_multipole_potential<<<(d.n_frag + 3) / 4, 128, 0, s>>>(d, cen, mult, pot);
    dim3 g((d.max_nao * d.max_nao + 127) / 128, d.n_frag);
    k_far_fock<<<g, 128, 0, s>>>(d, M, pot, nullptr, omega);
    note_launches(3);
    return cudaGetLastError();
}

cudaError_t launch_far_energy(const Dev& d, const double* E_far, double* E_frag, double* E_tot, cudaStream_t s)
{
    k_far_energy<<<1, 256, 0, s>>>(d, E_far, E_frag, E_tot);
    note_launches(1);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------ nuclear (Hermite)
// Field of the nuclei of fragment y on primitive pair P in Hermite form (McMurchie-Davidson):
//   V~_P[tuv] = sum_{C in y} -Z_C (2 pi/p) R_tuv(p, P - C),
// so that V^y_{mu nu} = sum_{P in (mu,nu)} K_P sum_tuv E^{mu nu}_tuv V~_P[tuv] and
// tr(D^x V^y) = sum_P sum_tuv Dtrue_P[tuv] V~_P[tuv] with Dtrue_P = Dh_P p/c (c = sqrt(2 pi^{5/2})).
template <int L>
__device__ __forceinline__ void nuclear_field(const Dev& d, const double4_32a P, int atom0, int nat, double (&acc)[nh(L)])
{
    double F[L + 1], base[L + 1], R[nh(L)];
    for (int c = atom0; c < atom0 + nat; ++c) {
        const double* C = d.atom_xyz + 3 * c;
        double X = P.x - C[0], Y = P.y - C[1], Z = P.z - C[2];
        double T = P.w * (X * X + Y * Y + Z * Z);
        boys_fp64<L>(d.boys, T, boys_row((float)T), F);
        double f = -d.atom_Z[c] * 2.0 * kPi / P.w;
#pragma unroll
        for (int n = 0; n <= L; ++n) {
            base[n] = f * F[n];
            f *= -2.0 * P.w;
        }
        md_R<L, double>(R, base, X, Y, Z);
#pragma unroll
        for (int k = 0; k < nh(L); ++k) acc[k] += R[k];
    }
}


// primitive pair number t of fragment x (classes in order) -> (class, global index in the class)
__device__ inline bool frag_prim_pair(const Dev& d, int x, int t, int& L, int& g)
{
    for (L = 0; L < kClasses; ++L) {
        int n = d.frag_npp[x * kClasses + L];
        if (t < n) {
            g = d.frag_pp0[x * kClasses + L] + t;
            return true;
        }
        t -= n;
    }
    return false;
}

// Environment field of all neighbours' nuclei on every primitive pair of x, in Hermite form,
// stored pre-scaled by p/c so that the J back-transform turns it into V_env.
template <int L>
__device__ __forceinline__ void nuclear_env_pp(const Dev& d, int x, int g, double* vh)
{
    const double4_32a P = d.pp_P[L][g];
    double acc[nh(L)];
#pragma unroll
    for (int k = 0; k < nh(L); ++k) acc[k] = 0.0;
    for (int c = d.frag_nbr0[x]; c < d.frag_nbr0[x + 1]; ++c) {
        const int y = d.nbr[c];
        nuclear_field<L>(d, P, d.frag_atom0[y], d.frag_nat[y], acc);
    }
    const double sc = P.w / kSqrt2Pi52;
#pragma unroll
    for (int k = 0; k < nh(L); ++k) vh[(size_t)k * d.n_pp[L] + g] = acc[k] * sc;
}

// The field of y's nuclei on primitive pair g of x, into its slot of the (pair, direction) block.
template <int L>
__device__ __forceinline__ void nuclear_trace_pp(const Dev& d, int x, int y, int g, int64_t base, double* fields)
{
    const double4_32a P = d.pp_P[L][g];
    double v[nh(L)];
#pragma unroll
    for (int k = 0; k < nh(L); ++k) v[k] = 0.0;
    nuclear_field<L>(d, P, d.frag_atom0[y], d.frag_nat[y], v);
    for (int L2 = 0; L2 < L; ++L2) base += (int64_t)nh(L2) * d.frag_npp[x * kClasses + L2];
    const int n = d.frag_npp[x * kClasses + L], i = g - d.frag_pp0[x * kClasses + L];
    const double sc = P.w / kSqrt2Pi52;
#pragma unroll
    for (int k = 0; k < nh(L); ++k) fields[base + (int64_t)k * n + i] = v[k] * sc;
}

__global__ void k_nuclear_env_h(Dev d, double* vh0, double* vh1, double* vh2, double* vh3, double* vh4)
{
    double* vh[kClasses] = {vh0, vh1, vh2, vh3, vh4};
    int x = blockIdx.y;
    int npp = 0;
    for (int L = 0; L < kClasses; ++L) npp += d.frag_npp[x * kClasses + L];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < npp; t += gridDim.x * blockDim.x) {
        int L, g;
        if (!frag_prim_pair(d, x, t, L, g)) continue;
        switch (L) {
            case 0: nuclear_env_pp<0>(d, x, g, vh[0]); break;
            case 1: nuclear_env_pp<1>(d, x, g, vh[1]); break;
            case 2: nuclear_env_pp<2>(d, x, g, vh[2]); break;
            case 3: nuclear_env_pp<3>(d, x, g, vh[3]); break;
            default: nuclear_env_pp<4>(d, x, g, vh[4]); break;
        }
    }
}

cudaError_t launch_nuclear_env(const Dev& d, double* vh[kClasses], double* V, cudaStream_t s)
{
    dim3 g(8, d.n_frag);
    k_nuclear_env_h<<<g, 128, 0, s>>>(d, vh[0], vh[1], vh[2], vh[3], vh[4]);
    note_launches(1);
    Dev dv = d;
    for (int L = 0; L < kClasses; ++L) dv.pp_Jh[L] = vh[L];
    return launch_back_transform(dv, V, s);
}

// tr(D^x V^y) for each pair, both directions: block (pair, direction), threads over the primitive
// pairs of the fragment whose electrons feel the other fragment's nuclei.
// tr[D^x V^y] for every pair and direction, V^y the attraction of y's nuclei, in two parts:
// geometry time: the Hermite field of y's nuclei on every primitive pair of x (pre-scaled by p/c
// so that it contracts directly with the stored Hermite density), stored per (pair, direction) at
// off[2 pair + dir], class after class, component-major as the Hermite densities;
// every build: tr = <Dh^x, field>, a dot product that reads the stored fields once.
__global__ void k_nuclear_trace_fields(Dev d, const int64_t* __restrict__ off, double* fields)
{
    const int pr = blockIdx.x, dir = blockIdx.y;
    const int x = dir == 0 ? d.pair_x[pr] : d.pair_y[pr];
    const int y = dir == 0 ? d.pair_y[pr] : d.pair_x[pr];
    int npp = 0;
    for (int L = 0; L < kClasses; ++L) npp += d.frag_npp[x * kClasses + L];
    for (int t = threadIdx.x; t < npp; t += blockDim.x) {
        int L, g;
        if (!frag_prim_pair(d, x, t, L, g)) continue;
        const int64_t base = off[2 * pr + dir];
        switch (L) {
            case 0: nuclear_trace_pp<0>(d, x, y, g, base, fields); break;
            case 1: nuclear_trace_pp<1>(d, x, y, g, base, fields); break;
            case 2: nuclear_trace_pp<2>(d, x, y, g, base, fields); break;
            case 3: nuclear_trace_pp<3>(d, x, y, g, base, fields); break;
            default: nuclear_trace_pp<4>(d, x, y, g, base, fields); break;
        }
    }
}

__global__ void k_nuclear_traces_dot(Dev d, const int64_t* __restrict__ off, const double* __restrict__ fields,
                                     double* tr_xy, double* tr_yx)
{
    const int pr = blockIdx.x, dir = blockIdx.y;
    const int x = dir == 0 ? d.pair_x[pr] : d.pair_y[pr];
    double acc = 0.0;
    int64_t base = off[2 * pr + dir];
    for (int L = 0; L < kClasses; ++L) {
        const int n = d.frag_npp[x * kClasses + L], g0 = d.frag_pp0[x * kClasses + L];
        for (int e = threadIdx.x; e < nh(L) * n; e += blockDim.x) {
            const int k = e / n, i = e % n;
            acc = fma(d.pp_Dh[L][(size_t)k * d.n_pp[L] + g0 + i], fields[base + e], acc);
        }
        base += (int64_t)nh(L) * n;
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        (dir == 0 ? tr_xy : tr_yx)[pr] = t;
    }
}

cudaError_t launch_nuclear_trace_fields(const Dev& d, const int64_t* off, double* fields, cudaStream_t s)
{
    if (d.n_pairs == 0) return cudaSuccess;
    k_nuclear_trace_fields<<<dim3(d.n_pairs, 2), 128, 0, s>>>(d, off, fields);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_nuclear_traces(const Dev& d, const int64_t* off, const double* fields, double* tr_xy,
                                  double* tr_yx, cudaStream_t s)
{
    if (d.n_pairs == 0) return cudaSuccess;
    k_nuclear_traces_dot<<<dim3(d.n_pairs, 2), 128, 0, s>>>(d, off, fields, tr_xy, tr_yx);
    note_launches(1);
    return cudaGetLastError();
}

// Nuclear repulsion: sum_{A<B in x} Z_A Z_B/R_AB per fragment, sum_{A in x, B in y} per pair.
__global__ void k_nuclear_repulsion(Dev d, double* e_intra, double* e_pair)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < d.n_frag) {
        double e = 0.0;
        int a0 = d.frag_atom0[i], na = d.frag_nat[i];
        for (int a = a0; a < a0 + na; ++a)
            for (int b = a0; b < a; ++b) {
                const double *A = d.atom_xyz + 3 * a, *B = d.atom_xyz + 3 * b;
                double r = sqrt((A[0] - B[0]) * (A[0] - B[0]) + (A[1] - B[1]) * (A[1] - B[1]) + (A[2] - B[2]) * (A[2] - B[2]));
                e += d.atom_Z[a] * d.atom_Z[b] / r;
            }
        e_intra[i] = e;
    }
    if (i < d.n_pairs) {
        int x = d.pair_x[i], y = d.pair_y[i];
        double e = 0.0;
        for (int a = d.frag_atom0[x]; a < d.frag_atom0[x] + d.frag_nat[x]; ++a)
            for (int b = d.frag_atom0[y]; b < d.frag_atom0[y] + d.frag_nat[y]; ++b) {
                const double *A = d.atom_xyz + 3 * a, *B = d.atom_xyz + 3 * b;
                double r = sqrt((A[0] - B[0]) * (A[0] - B[0]) + (A[1] - B[1]) * (A[1] - B[1]) + (A[2] - B[2]) * (A[2] - B[2]));
                e += d.atom_Z[a] * d.atom_Z[b] / r;
            }
        e_pair[i] = e;
    }
}

cudaError_t launch_nuclear_repulsion(const Dev& d, double* e_nn_intra, double* e_nn_pair, cudaStream_t s)
{
    int n = max(d.n_frag, d.n_pairs);
    k_nuclear_repulsion<<<(n + 127) / 128, 128, 0, s>>>(d, e_nn_intra, e_nn_pair);
    note_launches(1);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------ intra ERIs
// One thread per task = (fragment x, shell pairs s1 <= s2 of x, one bra component mu nu of s1):
// the row (mu nu|lambda sigma) for all lambda sigma of s2 by McMurchie-Davidson,
//   (mu nu|lambda sigma) = sum_{PQ} 2 pi^{5/2}/(p q sqrt(p+q)) sum_{tuv,t'u'v'} E^{mu nu}_{tuv}
//                          (-1)^{t'+u'+v'} E^{lambda sigma}_{t'u'v'} R_{t+t',u+u',v+v'}(alpha, PQ),
// written to the pair-packed tensor U[pq][rs] = (mu nu|lambda sigma), pq = pack(min(mu,nu),
// max(mu,nu)), np = n(n+1)/2 rows per fragment at frag_coff (both U[pq][rs] and U[rs][pq]).  Tasks
// are sorted by angular-momentum class so that the threads of a warp follow the same path.
// (mu nu|lambda sigma) for one bra Cartesian component kb of shell pair s1 (shells a <= b) and all
// components of shell pair s2 (c <= d), unnormalised primitives (ao_scale not applied):
// out[ic * ncart(ld) + id].  s1 and s2 may belong to different fragments.
__device__ void eri_bra_row(const Dev& d, const int s1, const int s2, const int kb, double* out)
{
    const int sa = d.sp_a[s1], sb = d.sp_b[s1], sc = d.sp_a[s2], sd = d.sp_b[s2];
    const int la = d.sh_l[sa], lb = d.sh_l[sb], lc = d.sh_l[sc], ld = d.sh_l[sd];
    const int nc = ncart(lc), nd = ncart(ld);
    const int L = la + lb + lc + ld;
    int ax, ay, az, bx, by, bz;
    cart_of(la, kb / ncart(lb), ax, ay, az);
    cart_of(lb, kb % ncart(lb), bx, by, bz);
    for (int k = 0; k < nc * nd; ++k) out[k] = 0.0;
    const double *A = d.atom_xyz + 3 * d.sh_atom[sa], *B = d.atom_xyz + 3 * d.sh_atom[sb];
    const double *C = d.atom_xyz + 3 * d.sh_atom[sc], *Dc = d.atom_xyz + 3 * d.sh_atom[sd];
    double AB2 = 0, CD2 = 0;
    for (int k = 0; k < 3; ++k) {
        AB2 += (A[k] - B[k]) * (A[k] - B[k]);
        CD2 += (C[k] - Dc[k]) * (C[k] - Dc[k]);
    }
    int kc[36][3];
    for (int ic = 0; ic < nc; ++ic)
        for (int id = 0; id < nd; ++id) {
            int cx, cy, cz, dx, dy, dz;
            cart_of(lc, ic, cx, cy, cz);
            cart_of(ld, id, dx, dy, dz);
            kc[ic * nd + id][0] = cx * 8 + dx;  // packed (c, d) exponent pairs per direction
            kc[ic * nd + id][1] = cy * 8 + dy;
            kc[ic * nd + id][2] = cz * 8 + dz;
        }
    for (int i = 0; i < d.sh_np[sa]; ++i)
        for (int j = 0; j < d.sh_np[sb]; ++j) {
            double a = d.p_exp[d.sh_p0[sa] + i], b = d.p_exp[d.sh_p0[sb] + j], p = a + b;
            double Kab = d.p_coef[d.sh_p0[sa] + i] * d.p_coef[d.sh_p0[sb] + j] * exp(-a * b / p * AB2);
            double P[3], Eb[3][5];
            for (int k = 0; k < 3; ++k) P[k] = (a * A[k] + b * B[k]) / p;
            {
                double E[3][3][5];
                md_E1(ax, bx, p, P[0] - A[0], P[0] - B[0], E);
                for (int t = 0; t < 5; ++t) Eb[0][t] = t <= ax + bx ? E[ax][bx][t] : 0.0;
                md_E1(ay, by, p, P[1] - A[1], P[1] - B[1], E);
                for (int t = 0; t < 5; ++t) Eb[1][t] = t <= ay + by ? E[ay][by][t] : 0.0;
                md_E1(az, bz, p, P[2] - A[2], P[2] - B[2], E);
                for (int t = 0; t < 5; ++t) Eb[2][t] = t <= az + bz ? E[az][bz][t] : 0.0;
            }
            for (int k2 = 0; k2 < d.sh_np[sc]; ++k2)
                for (int l2 = 0; l2 < d.sh_np[sd]; ++l2) {
                    double c = d.p_exp[d.sh_p0[sc] + k2], e = d.p_exp[d.sh_p0[sd] + l2], q = c + e;
                    double Kcd = d.p_coef[d.sh_p0[sc] + k2] * d.p_coef[d.sh_p0[sd] + l2] * exp(-c * e / q * CD2);
                    double Q[3], Ek[3][3][3][5];
                    for (int k = 0; k < 3; ++k) {
                        Q[k] = (c * C[k] + e * Dc[k]) / q;
                        md_E1(lc, ld, q, Q[k] - C[k], Q[k] - Dc[k], Ek[k]);
                    }
                    double alpha = p * q / (p + q);
                    double X = P[0] - Q[0], Y = P[1] - Q[1], Z = P[2] - Q[2];
                    double F[kMaxLTot + 1], base[kMaxLTot + 1], R[nh(kMaxLTot)];
                    boys_fp64_rt(d.boys, alpha * (X * X + Y * Y + Z * Z), L, F);
                    double pre = kSqrt2Pi52 * kSqrt2Pi52 / (p * q * sqrt(p + q)) * Kab * Kcd;  // 2 pi^{5/2}
                    for (int m = 0; m <= L; ++m) {
                        base[m] = pre * F[m];
                        pre *= -2.0 * alpha;
                    }
                    md_R_rt(L, R, base, X, Y, Z);
                    // Ybra[t'u'v'] = sum_tuv Eb R[t+t', ...]
                    double Yb[nh(2 * kMaxL)];
                    const int LCD = lc + ld;
                    for (int h = 0; h < nh(LCD); ++h) {
                        TUV c2 = htuv(h);
                        double y = 0.0;
                        for (int t = 0; t <= ax + bx; ++t)
                            for (int u = 0; u <= ay + by; ++u)
                                for (int v = 0; v <= az + bz; ++v)
                                    y += Eb[0][t] * Eb[1][u] * Eb[2][v] * R[hidx(t + c2.t, u + c2.u, v + c2.v)];
                        Yb[h] = ((c2.t + c2.u + c2.v) & 1) ? -y : y;
                    }
                    for (int k = 0; k < nc * nd; ++k) {
                        int cx = kc[k][0] >> 3, dx = kc[k][0] & 7, cy = kc[k][1] >> 3, dy = kc[k][1] & 7;
                        int cz = kc[k][2] >> 3, dz = kc[k][2] & 7;
                        double v = 0.0;
                        for (int t = 0; t <= cx + dx; ++t)
                            for (int u = 0; u <= cy + dy; ++u)
                                for (int vv = 0; vv <= cz + dz; ++vv)
                                    v += Ek[0][cx][dx][t] * Ek[1][cy][dy][u] * Ek[2][cz][dz][vv] * Yb[hidx(t, u, vv)];
                        out[k] += v;
                    }
                }
        }
}

// The same row for shells of angular momenta known at compile time (s and p: 16 classes), from the
// primitive-pair data of the J-engine (P, p, K = c_i c_j exp(-ab/p |AB|^2)): the bra component's
// Hermite coefficients and the ket's, the Boys function, R recursion and both contractions in
// registers, no transcendental per primitive quartet but one reciprocal square root.
// Picks E[ai][bi][t] of the (LA+1) x (LB+1) table for runtime ai, bi with compile-time indices.
template <int LA, int LB>
__device__ __forceinline__ double e_pick(const double (*E)[3][5], int ai, int bi, int t)
{
    double v = 0.0;
#pragma unroll
    for (int i = 0; i <= LA; ++i)
#pragma unroll
        for (int j = 0; j <= LB; ++j)
            if (i == ai && j == bi) v = E[i][j][t];
    return v;
}

// Lane `sub` of the nsub lanes that share one task takes the primitive quartets sub, sub + nsub, ...
// (its partial rows in out[NKB][NC ND]; the caller sums the lanes).
template <int LA, int LB, int LC, int LD, int NKB>
__device__ __forceinline__ void eri_bra_row_t(const Dev& d, const int s1, const int s2, const int kb0, double* out,
                                              const int sub, const int nsub)
{
    constexpr int NBc = ncart(LB), NC = ncart(LC), ND = ncart(LD), NK = NC * ND;
    constexpr int LAB = LA + LB, LCD = LC + LD, L = LAB + LCD;
    const int sa = d.sp_a[s1], sb = d.sp_b[s1], sc = d.sp_a[s2], sd = d.sp_b[s2];
    int ax[NKB], ay[NKB], az[NKB], bx[NKB], by[NKB], bz[NKB];
#pragma unroll
    for (int j = 0; j < NKB; ++j) {
        cart_of(LA, (kb0 + j) / NBc, ax[j], ay[j], az[j]);
        cart_of(LB, (kb0 + j) % NBc, bx[j], by[j], bz[j]);
    }
    const double *A = d.atom_xyz + 3 * d.sh_atom[sa], *B = d.atom_xyz + 3 * d.sh_atom[sb];
    const double *C = d.atom_xyz + 3 * d.sh_atom[sc], *Dc = d.atom_xyz + 3 * d.sh_atom[sd];
#pragma unroll
    for (int k = 0; k < NKB * NK; ++k) out[k] = 0.0;
    const int gP0 = d.sp_pp0[s1], nP = d.sh_np[sa] * d.sh_np[sb];
    const int gQ0 = d.sp_pp0[s2], nQ = d.sh_np[sc] * d.sh_np[sd];
    for (int pq = sub; pq < nP * nQ; pq += nsub) {
        const int i = pq % nP, j = pq / nP;
        const double4_32a Q = d.pp_P[LCD][gQ0 + j];
        const double q = Q.w;
        const double cq = d.pp_K[LCD][gQ0 + j] * kSqrt2Pi52 / q;
        double Ek[3][3][3][5];
        md_E1(LC, LD, q, Q.x - C[0], Q.x - Dc[0], Ek[0]);
        md_E1(LC, LD, q, Q.y - C[1], Q.y - Dc[1], Ek[1]);
        md_E1(LC, LD, q, Q.z - C[2], Q.z - Dc[2], Ek[2]);
        {
            const double4_32a P = d.pp_P[LAB][gP0 + i];
            const double p = P.w;
            const double cp = d.pp_K[LAB][gP0 + i] * kSqrt2Pi52 / p;
            double Ea[3][3][3][5];
            md_E1(LA, LB, p, P.x - A[0], P.x - B[0], Ea[0]);
            md_E1(LA, LB, p, P.y - A[1], P.y - B[1], Ea[1]);
            md_E1(LA, LB, p, P.z - A[2], P.z - B[2], Ea[2]);
            const double X = P.x - Q.x, Y = P.y - Q.y, Z = P.z - Q.z;
            const double rs = rsqrt(p + q);
            const double alpha = p * q * (rs * rs);
            const double T = alpha * (X * X + Y * Y + Z * Z);
            double F[L + 1], base[L + 1], R[nh(L)];
            boys_fp64<L>(d.boys, T, boys_row((float)T), F);
            double pre = cp * cq * rs;
#pragma unroll
            for (int m = 0; m <= L; ++m) {
                base[m] = pre * F[m];
                pre *= -2.0 * alpha;
            }
            md_R<L, double>(R, base, X, Y, Z);
#pragma unroll
            for (int jb = 0; jb < NKB; ++jb) {
            double Eb[3][LAB + 1];
#pragma unroll
            for (int t = 0; t <= LAB; ++t) {
                Eb[0][t] = e_pick<LA, LB>(Ea[0], ax[jb], bx[jb], t);
                Eb[1][t] = e_pick<LA, LB>(Ea[1], ay[jb], by[jb], t);
                Eb[2][t] = e_pick<LA, LB>(Ea[2], az[jb], bz[jb], t);
            }
            double Yb[nh(LCD)];
            static_for<nh(LCD)>([&](auto H) {
                constexpr TUV c2 = htuv(decltype(H)::value);
                double y = 0.0;
#pragma unroll
                for (int t = 0; t <= LAB; ++t)
#pragma unroll
                    for (int u = 0; u <= LAB - t; ++u)
#pragma unroll
                        for (int v = 0; v <= LAB - t - u; ++v)
                            if (t <= ax[jb] + bx[jb] && u <= ay[jb] + by[jb] && v <= az[jb] + bz[jb])
                                y += Eb[0][t] * Eb[1][u] * Eb[2][v] * R[hidx(t + c2.t, u + c2.u, v + c2.v)];
                Yb[decltype(H)::value] = ((c2.t + c2.u + c2.v) & 1) ? -y : y;
            });
#pragma unroll
            for (int ic = 0; ic < NC; ++ic) {
                int cx, cy, cz;
                cart_of(LC, ic, cx, cy, cz);
#pragma unroll
                for (int id = 0; id < ND; ++id) {
                    int dx, dy, dz;
                    cart_of(LD, id, dx, dy, dz);
                    double v = 0.0;
#pragma unroll
                    for (int t = 0; t <= LCD; ++t)
#pragma unroll
                        for (int u = 0; u <= LCD - t; ++u)
#pragma unroll
                            for (int w = 0; w <= LCD - t - u; ++w)
                                if (t <= cx + dx && u <= cy + dy && w <= cz + dz)
                                    v += e_pick<LC, LD>(Ek[0], cx, dx, t) * e_pick<LC, LD>(Ek[1], cy, dy, u) *
                                         e_pick<LC, LD>(Ek[2], cz, dz, w) * Yb[hidx(t, u, w)];
                    out[jb * NK + ic * ND + id] += v;
                }
            }
            }
        }
    }
}

// Writes the row of task w (fragment x, shell pairs s1 <= s2, bra component kb) into U[pq][rs] and
// U[rs][pq], scaled to normalised AOs (NC, ND > 0: the ket shells' component counts at compile time).
template <int NC = 0, int ND = 0>
__device__ __forceinline__ void intra_eri_store(const Dev& d, const int4 tk, const double* out, double* eri)
{
    const int x = tk.x, s1 = tk.y, s2 = tk.z, kb = tk.w;
    const int sa = d.sp_a[s1], sb = d.sp_b[s1], sc = d.sp_a[s2], sd = d.sp_b[s2];
    const int lb = d.sh_l[sb];
    const int nc = NC > 0 ? NC : ncart(d.sh_l[sc]), nd = ND > 0 ? ND : ncart(d.sh_l[sd]);
    const int n = d.frag_nao[x];
    const int ao0 = d.frag_ao0[x];
    const int64_t np = (int64_t)n * (n + 1) / 2;
    double* U = eri + d.frag_coff[x];
    const int mu = d.sh_ao[sa] + kb / ncart(lb), nu = d.sh_ao[sb] + kb % ncart(lb);
    const double smn = d.ao_scale[ao0 + mu] * d.ao_scale[ao0 + nu];
    const int64_t pq = pair_pack(mu, nu, n);
#pragma unroll
    for (int k = 0; k < (NC > 0 ? NC * ND : 36); ++k) {
        if (NC == 0 && k >= nc * nd) break;
        int la_ = d.sh_ao[sc] + k / nd, si = d.sh_ao[sd] + k % nd;
        double v = out[k] * smn * d.ao_scale[ao0 + la_] * d.ao_scale[ao0 + si];
        const int64_t rs = pair_pack(la_, si, n);
        U[pq * np + rs] = v;
        U[rs * np + pq] = v;
    }
}

// kIntraLanes lanes per task (the primitive quartets split between them, partial rows summed by a
// butterfly over the lane group in a fixed order).
constexpr int kIntraLanes = 8;

template <int LA, int LB, int LC, int LD>
__global__ void __launch_bounds__(128) k_intra_eri_t(Dev d, const int4* __restrict__ tasks, int n_tasks, double* eri)
{
    constexpr int NK = ncart(LC) * ncart(LD), NKB = intra_nkb(LA, LB, LC, LD);
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) / kIntraLanes, sub = threadIdx.x % kIntraLanes;
    const bool on = w < n_tasks;  // whole lane groups (128 is a multiple of kIntraLanes)
    const int4 tk = tasks[on ? w : 0];
    double out[NKB * NK];
    if (on) eri_bra_row_t<LA, LB, LC, LD, NKB>(d, tk.y, tk.z, tk.w, out, sub, kIntraLanes);
#pragma unroll
    for (int k = 0; k < NKB * NK; ++k) {
        if (!on) out[k] = 0.0;
#pragma unroll
        for (int o = kIntraLanes / 2; o > 0; o >>= 1) out[k] += __shfl_xor_sync(0xffffffffu, out[k], o, kIntraLanes);
    }
    if (on && sub == 0)
#pragma unroll
        for (int j = 0; j < NKB; ++j)
            intra_eri_store<ncart(LC), ncart(LD)>(d, make_int4(tk.x, tk.y, tk.z, tk.w + j), out + j * NK, eri);
}

__global__ void k_intra_eri(Dev d, const int4* __restrict__ tasks, int n_tasks, double* eri)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= n_tasks) return;
    const int4 tk = tasks[w];
    double out[36];
    eri_bra_row(d, tk.y, tk.z, tk.w, out);
    intra_eri_store<>(d, tk, out, eri);
}

template <int LA, int LB, int LC, int LD>
void launch_intra_class(const Dev& d, const int4* tasks, int n, double* eri, cudaStream_t s)
{
    k_intra_eri_t<LA, LB, LC, LD><<<(unsigned)(((int64_t)n * kIntraLanes + 127) / 128), 128, 0, s>>>(d, tasks, n, eri);
}

// The class launches are small (a few hundred blocks each on the water workloads): they run on the
// context stream and two side streams, forked and joined by events, the largest classes first, each
// on the stream with the least work so far.
cudaError_t launch_intra_eri(const Dev& d, const int4* tasks, const std::vector<int>& cls_off, double* eri,
                             cudaStream_t s)
{
    constexpr int kStreams = 3;
    std::vector<std::pair<double, int>> order;
    for (int cls = 0; cls + 1 < (int)cls_off.size(); ++cls) {
        const int n = cls_off[cls + 1] - cls_off[cls];
        if (n <= 0) continue;
        const int la = cls / 27, lb = (cls / 9) % 3, lc = (cls / 3) % 3, ld = cls % 3;
        const double w = (double)n * ncart(lc) * ncart(ld) * (1 + la + lb + lc + ld);  // rough cost
        order.push_back({-w, cls});
    }
    std::sort(order.begin(), order.end());
    cudaStream_t st[kStreams] = {s, nullptr, nullptr};
    cudaEvent_t fork = nullptr, join[kStreams] = {};
    cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    for (int i = 1; i < kStreams && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&st[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventRecord(fork, s);
    for (int i = 1; i < kStreams && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(st[i], fork, 0);
    double load[kStreams] = {};
    for (size_t o = 0; o < order.size() && e == cudaSuccess; ++o) {
        const int cls = order[o].second;
        const int n = cls_off[cls + 1] - cls_off[cls];
        int si = 0;
        for (int i = 1; i < kStreams; ++i)
            if (load[i] < load[si]) si = i;
        load[si] -= order[o].first;
        const cudaStream_t sc = st[si];
        const int4* t = tasks + cls_off[cls];
        const int la = cls / 27, lb = (cls / 9) % 3, lc = (cls / 3) % 3, ld = cls % 3;
        if (la > 1 || lb > 1 || lc > 1 || ld > 1) {
            k_intra_eri<<<(n + 127) / 128, 128, 0, sc>>>(d, t, n, eri);
        } else {
            switch (la * 8 + lb * 4 + lc * 2 + ld) {
#define FEF_IE(A, B, C, D) \
    case A * 8 + B * 4 + C * 2 + D: launch_intra_class<A, B, C, D>(d, t, n, eri, sc); break;
                FEF_IE(0, 0, 0, 0) FEF_IE(0, 0, 0, 1) FEF_IE(0, 0, 1, 0) FEF_IE(0, 0, 1, 1)
                FEF_IE(0, 1, 0, 0) FEF_IE(0, 1, 0, 1) FEF_IE(0, 1, 1, 0) FEF_IE(0, 1, 1, 1)
                FEF_IE(1, 0, 0, 0) FEF_IE(1, 0, 0, 1) FEF_IE(1, 0, 1, 0) FEF_IE(1, 0, 1, 1)
                FEF_IE(1, 1, 0, 0) FEF_IE(1, 1, 0, 1) FEF_IE(1, 1, 1, 0) FEF_IE(1, 1, 1, 1)
#undef FEF_IE
                default: break;
            }
        }
        note_launches(1);
        e = cudaGetLastError();
    }
    // join the side streams into s (also after an error, so that no work is left unordered)
    for (int i = 1; i < kStreams; ++i) {
        if (!st[i]) continue;
        if (join[i] && cudaEventRecord(join[i], st[i]) == cudaSuccess) cudaStreamWaitEvent(s, join[i], 0);
        cudaStreamDestroy(st[i]);
        if (join[i]) cudaEventDestroy(join[i]);
    }
    if (fork) cudaEventDestroy(fork);
    return e != cudaSuccess ? e : cudaGetLastError();
}

// Inter-fragment blocks for a list of fragment pairs: task (list position q, s1 in x, s2 in y, kb),
// W_q[pq][rs] = (mu nu|lambda sigma), pq = pair(mu <= nu) over x's AOs, rs = pair(lambda <= sigma)
// over y's AOs, at off[q] (np_x * np_y doubles per pair).
__global__ void k_pair_eri(Dev d, const int4* __restrict__ tasks, int n_tasks, const int* __restrict__ pair_of,
                           const int64_t* __restrict__ off, double* W)
{
    int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= n_tasks) return;
    const int4 tk = tasks[w];
    const int q = tk.x, s1 = tk.y, s2 = tk.z, kb = tk.w;
    const int pr = pair_of[q];
    const int x = d.pair_x[pr], y = d.pair_y[pr];
    const int sa = d.sp_a[s1], sb = d.sp_b[s1], sc = d.sp_a[s2], sd = d.sp_b[s2];
    const int lb = d.sh_l[sb];
    const int nc = ncart(d.sh_l[sc]), nd = ncart(d.sh_l[sd]);
    double out[36];
    eri_bra_row(d, s1, s2, kb, out);
    const int nx = d.frag_nao[x], ny = d.frag_nao[y];
    const int64_t npy = (int64_t)ny * (ny + 1) / 2;
    const int mu = d.sh_ao[sa] + kb / ncart(lb), nu = d.sh_ao[sb] + kb % ncart(lb);
    const double smn = d.ao_scale[d.frag_ao0[x] + mu] * d.ao_scale[d.frag_ao0[x] + nu];
    const int64_t pq = pair_pack(mu, nu, nx);
    double* Wq = W + off[q];
    for (int k = 0; k < nc * nd; ++k) {
        const int la_ = d.sh_ao[sc] + k / nd, si = d.sh_ao[sd] + k % nd;
        Wq[pq * npy + pair_pack(la_, si, ny)] =
            out[k] * smn * d.ao_scale[d.frag_ao0[y] + la_] * d.ao_scale[d.frag_ao0[y] + si];
    }
}

cudaError_t launch_pair_eri(const Dev& d, const int4* tasks, int n_tasks, const int* pair_of, const int64_t* off,
                            double* W, cudaStream_t s)
{
    if (n_tasks > 0) {
        k_pair_eri<<<(n_tasks + 127) / 128, 128, 0, s>>>(d, tasks, n_tasks, pair_of, off, W);
        note_launches(1);
    }
    return cudaGetLastError();
}

// Coulomb-minus-half-exchange tensor, so that G[D] = J[D] - K[D]/2 is one contraction:
//   C[mu nu][lambda sigma] = (mu nu|lambda sigma) - (1/2) (mu lambda|nu sigma).
// Stored packed over mu <= nu and lambda <= sigma (D and G are symmetric) and transposed:
//   CT[rs][pq] = C[mu nu][lambda sigma] + [lambda != sigma] C[mu nu][sigma lambda],
// with pq = pair(mu, nu), rs = pair(lambda, sigma), pair(i, j) = i n - i (i - 1)/2 + (j - i), i <= j,
// so that G_pq = sum_rs CT[rs][pq] D_rs and a warp of consecutive pq reads consecutive doubles.
__device__ inline int tri_i(int p, int n)
{
    int i = 0;
    while (p >= n - i) { p -= n - i; ++i; }
    return i;
}

// CT[rs][pq] = (mu nu|la si) - (mu la|nu si)/2 + [la != si] ((mu nu|si la) - (mu si|nu la)/2) from the
// pair-packed U, so that G[D]_{mu nu} = sum_{rs} CT[rs][pq] D_{la si} over la <= si.
__global__ void k_coulomb_exchange(Dev d, const double* eri, double* eric)
{
    int x = blockIdx.y;
    int n = d.frag_nao[x];
    int64_t np = (int64_t)n * (n + 1) / 2;
    const double* U = eri + d.frag_coff[x];
    double* c = eric + d.frag_coff[x];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < np * np; i += (int64_t)gridDim.x * blockDim.x) {
        int rs = (int)(i / np), pq = (int)(i % np);
        int mu = tri_i(pq, n), nu = mu + pq - (mu * n - mu * (mu - 1) / 2);
        int la = tri_i(rs, n), si = la + rs - (la * n - la * (la - 1) / 2);
        double v = U[(int64_t)pq * np + rs] - 0.5 * U[pair_pack(mu, la, n) * np + pair_pack(nu, si, n)];
        if (la != si) v += U[(int64_t)pq * np + rs] - 0.5 * U[pair_pack(mu, si, n) * np + pair_pack(nu, la, n)];
        c[i] = v;
    }
}

cudaError_t launch_coulomb_exchange(const Dev& d, const double* eri, double* eric, cudaStream_t s)
{
    size_t npm = (size_t)d.max_nao * (d.max_nao + 1) / 2;
    size_t n4 = npm * npm;
    dim3 g((unsigned)std::min<size_t>((n4 + 255) / 256, 8192), d.n_frag);
    k_coulomb_exchange<<<g, 256, 0, s>>>(d, eri, eric);
    note_launches(1);
    return cudaGetLastError();
}

// Schwarz factors Q_ab = max_{mu in a, nu in b} sqrt|(mu nu|mu nu)| from the intra tensor; each
// primitive pair of the shell pair gets a float copy for the J-engine's screening test.
__global__ void k_schwarz(Dev d, const double* eri, double* sp_Q, float* pq0, float* pq1, float* pq2, float* pq3,
                          float* pq4)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= d.n_sp) return;
    int sa = d.sp_a[s], sb = d.sp_b[s];
    int x = 0;
    {  // fragment of the shell pair: binary search over frag_sp0
        int lo = 0, hi = d.n_frag - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) / 2;
            if (d.frag_sp0[mid] <= s) lo = mid; else hi = mid - 1;
        }
        x = lo;
    }
    int n = d.frag_nao[x];
    const int64_t np = (int64_t)n * (n + 1) / 2;
    const double* U = eri + d.frag_coff[x];
    double q = 0.0;
    for (int ia = 0; ia < ncart(d.sh_l[sa]); ++ia)
        for (int ib = 0; ib < ncart(d.sh_l[sb]); ++ib) {
            int mu = d.sh_ao[sa] + ia, nu = d.sh_ao[sb] + ib;
            const int64_t mn = pair_pack(mu, nu, n);
            q = fmax(q, fabs(U[mn * np + mn]));
        }
    q = sqrt(q);
    sp_Q[s] = q;
    float* pq[kClasses] = {pq0, pq1, pq2, pq3, pq4};
    int L = d.sp_L[s];
    const int npp = d.sh_np[sa] * d.sh_np[sb];
    for (int k = 0; k < npp; ++k) pq[L][d.sp_pp0[s] + k] = (float)q;
}

cudaError_t launch_schwarz(const Dev& d, const double* eri, double* sp_Q, float* pp_Q[kClasses], cudaStream_t s)
{
    k_schwarz<<<(d.n_sp + 127) / 128, 128, 0, s>>>(d, eri, sp_Q, pp_Q[0], pp_Q[1], pp_Q[2], pp_Q[3], pp_Q[4]);
    note_launches(1);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------ neighbours
// flags[x * n_frag + y] = 1 for y > x when min_{A in x, B in y} |R_A - R_B| < cutoff (bohr).
__global__ void k_neighbours(Dev d, double cutoff, unsigned char* flags)
{
    int x = blockIdx.y;
    for (int y = x + 1 + blockIdx.x * blockDim.x + threadIdx.x; y < d.n_frag; y += gridDim.x * blockDim.x) {
        double best = 1e300;
        for (int a = d.frag_atom0[x]; a < d.frag_atom0[x] + d.frag_nat[x]; ++a)
            for (int b = d.frag_atom0[y]; b < d.frag_atom0[y] + d.frag_nat[y]; ++b) {
                const double *A = d.atom_xyz + 3 * a, *B = d.atom_xyz + 3 * b;
                double r2 = (A[0] - B[0]) * (A[0] - B[0]) + (A[1] - B[1]) * (A[1] - B[1]) + (A[2] - B[2]) * (A[2] - B[2]);
                best = fmin(best, r2);
            }
        flags[(size_t)x * d.n_frag + y] = (cutoff <= 0.0 || best < cutoff * cutoff) ? 1 : 0;
    }
}

cudaError_t launch_neighbours(const Dev& d, double cutoff_bohr, unsigned char* flags, cudaStream_t s)
{
    dim3 g((d.n_frag + 255) / 256, d.n_frag);
    k_neighbours<<<g, 256, 0, s>>>(d, cutoff_bohr, flags);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace fef
