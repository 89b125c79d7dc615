// Fragment RHF in a frozen environment field (paper, "Fragment Mean Field": each fragment's
// determinant satisfies the Hartree-Fock equation with F~ = h(1) + (2J - K) + omega_x; the
// fragment orbitals are orthonormal in the fragment's own overlap metric S^x).
//
// One thread block per fragment runs the whole micro-iteration loop on the device:
//   G = C D (C: Coulomb-minus-half-exchange tensor), F = h + omega + G,
//   E_scf = tr[D (h + omega + F)]/2 + E_nn, e = F D S - S D F,
//   Pulay DIIS on X^T e X, F' = X^T F X, cyclic Jacobi eigensolver, aufbau, D = 2 C_occ C_occ^T,
// until |dE_scf| < e_tol and max|e| < comm_tol.  X = U s^{-1/2} is the canonical orthogonaliser.
#include <cooperative_groups.h>

#include "common.cuh"
#include "internal.hpp"

namespace fef {

namespace {

namespace cg = cooperative_groups;

// The threads that share one fragment's micro loop: one thread block (CS = 1), or the CS blocks of a
// thread-block cluster (fragments above the shared-memory limit, matrices in global memory).  Loops
// over matrix elements are spread over all CS * blockDim threads; sync() orders the phases (a
// cluster barrier, release/acquire at cluster scope, for CS > 1).  Every block of a cluster takes
// the same control-flow decisions: the reductions that feed them are summed in the same order.
template <int CS>
struct Team {
    int rank;
    __device__ __forceinline__ int g() const { return rank * (int)blockDim.x + (int)threadIdx.x; }
    __device__ __forceinline__ int gs() const { return CS * (int)blockDim.x; }
    __device__ __forceinline__ void sync() const
    {
        if constexpr (CS == 1)
            __syncthreads();
        else
            cg::this_cluster().sync();
    }
};

// Team-wide sum (MAX = false) or maximum; red: 40 doubles of shared memory.
template <int CS, bool MAX>
__device__ double team_reduce(const Team<CS>& t, double v, double* red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double u = __shfl_xor_sync(0xffffffffu, v, o);
        v = MAX ? fmax(v, u) : v + u;
    }
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s = MAX ? fmax(s, red[w]) : s + red[w];
        red[32] = s;
    }
    if constexpr (CS == 1) {
        __syncthreads();
        const double r = red[32];
        __syncthreads();
        return r;
    } else {
        cg::cluster_group cl = cg::this_cluster();
        cl.sync();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int r = 0; r < CS; ++r) {
                const double u = *cl.map_shared_rank(red + 32, r);
                s = MAX ? fmax(s, u) : s + u;
            }
            red[33] = s;
        }
        cl.sync();
        return red[33];
    }
}

template <int CS>
__device__ inline double team_sum(const Team<CS>& t, double v, double* red) { return team_reduce<CS, false>(t, v, red); }
template <int CS>
__device__ inline double team_max(const Team<CS>& t, double v, double* red) { return team_reduce<CS, true>(t, v, red); }

// C[m x k] = op(A) B with A, B, C row-major, leading dimension ld.
// transA: C = A^T B with A stored k x m.
template <int CS>
__device__ inline void mm(const Team<CS>& t, double* C, const double* A, const double* B, int m, int k, int ncol,
                          int ld, bool transA)
{
    for (int e = t.g(); e < m * ncol; e += t.gs()) {
        int i = e / ncol, j = e % ncol;
        double s = 0.0;
        if (transA)
            for (int l = 0; l < k; ++l) s = fma(A[l * ld + i], B[l * ld + j], s);
        else
            for (int l = 0; l < k; ++l) s = fma(A[i * ld + l], B[l * ld + j], s);
        C[i * ld + j] = s;
    }
    t.sync();
}

struct JacobiScratch {
    double c[kMaxFragAO / 2], s[kMaxFragAO / 2];
    int p[kMaxFragAO / 2], q[kMaxFragAO / 2];
};

// Cyclic Jacobi on the symmetric m x m matrix A (shared or global, leading dimension ld),
// m <= kMaxFragAO.
// Parallel ordering: round-robin pairing (circle method), m/2 disjoint rotations per round, each
// zeroing A_pq with t = sgn(theta)/(|theta| + sqrt(theta^2 + 1)), theta = (A_qq - A_pp)/(2 A_pq)
// (Golub & Van Loan, symmetric Schur decomposition).  Every block of the team computes the rotations
// of a round itself (into its own scratch); row updates, then column updates, are spread over the team.
// On exit diag(A) holds the eigenvalues and the columns of V the eigenvectors.  Stops when the
// off-diagonal Frobenius norm is below 1e-12 times the largest diagonal magnitude (eigenvalue errors
// of order 1e-24 relative, eigenvector errors of 1e-12, far below the SCF commutator threshold).
template <int CS>
__device__ void jacobi_eigh(const Team<CS>& t, double* A, double* V, int m, int ld, JacobiScratch* js, double* red)
{
    // A built from matrix products is symmetric only to rounding; an orthogonal similarity keeps
    // the antisymmetric part, so symmetrise first and measure convergence on the upper triangle.
    for (int e = t.g(); e < m * m; e += t.gs()) {
        int r = e / m, c = e % m;
        V[r * ld + c] = (r == c) ? 1.0 : 0.0;
        if (r < c) {
            double v = 0.5 * (A[r * ld + c] + A[c * ld + r]);
            A[r * ld + c] = v;
            A[c * ld + r] = v;
        }
    }
    t.sync();
    const int M = m + (m & 1);
    const int half = M / 2;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, dg = 0.0;
        for (int e = t.g(); e < m * m; e += t.gs()) {
            int r = e / m, c = e % m;
            double v = A[r * ld + c];
            if (r < c) off += 2.0 * v * v; else if (r == c) dg = fmax(dg, fabs(v));
        }
        off = team_sum(t, off, red);
        dg = team_max(t, dg, red);
        if (off <= 1e-24 * fmax(dg * dg, 1e-300)) break;
        for (int rnd = 0; rnd < M - 1; ++rnd) {
            for (int k = threadIdx.x; k < half; k += blockDim.x) {
                int i1 = (k == 0) ? 0 : ((k - 1 + rnd) % (M - 1)) + 1;
                int k2 = M - 1 - k;
                int i2 = ((k2 - 1 + rnd) % (M - 1)) + 1;
                int p = min(i1, i2), q = max(i1, i2);
                double c = 1.0, s = 0.0;
                if (q < m) {
                    // rotation angle in FP32 (any exact rotation reduces A_pq; FP32 t leaves a 1e-7
                    // residual that the next sweep removes); c and s in FP64 so c^2 + s^2 = 1
                    const float apq = (float)A[p * ld + q];
                    if (apq != 0.0f) {
                        const float theta = (float)(A[q * ld + q] - A[p * ld + p]) / (2.0f * apq);
                        float tt = 1.0f / (fabsf(theta) + sqrtf(fmaf(theta, theta, 1.0f)));
                        if (theta < 0.0f) tt = -tt;
                        const double td = (double)tt;
                        c = rsqrt(fma(td, td, 1.0));
                        s = td * c;
                    }
                }
                js->p[k] = p;
                js->q[k] = q;
                js->c[k] = c;
                js->s[k] = s;
            }
            // every block has read the A entries of this round before any row is rewritten
            if constexpr (CS == 1) __syncthreads(); else t.sync();
            for (int w = t.g(); w < half * m; w += t.gs()) {
                int k = w / m, j = w % m;
                int p = js->p[k], q = js->q[k];
                if (q >= m || js->s[k] == 0.0) continue;
                double c = js->c[k], s = js->s[k];
                double ap = A[p * ld + j], aq = A[q * ld + j];
                A[p * ld + j] = c * ap - s * aq;
                A[q * ld + j] = s * ap + c * aq;
            }
            t.sync();
            for (int w = t.g(); w < half * m; w += t.gs()) {
                int k = w / m, i = w % m;
                int p = js->p[k], q = js->q[k];
                if (q >= m || js->s[k] == 0.0) continue;
                double c = js->c[k], s = js->s[k];
                double ap = A[i * ld + p], aq = A[i * ld + q];
                A[i * ld + p] = c * ap - s * aq;
                A[i * ld + q] = s * ap + c * aq;
                double vp = V[i * ld + p], vq = V[i * ld + q];
                V[i * ld + p] = c * vp - s * vq;
                V[i * ld + q] = s * vp + c * vq;
            }
            t.sync();
        }
    }
}


// ------------------------------------------------------------------------------------------ E_M2
// Monomer second-order energy (Eq. EM2 with the first-order doubles of Eq. monDoubles) of each
// fragment on its canonical FEF orbitals: F C = S C eps (canonical orthogonaliser X, cyclic Jacobi,
// ascending order, aufbau), (ia|jb) = sum C_mu i C_nu a C_lambda j C_sigma b (mu nu|lambda sigma) by
// four quarter-transforms of the pair-packed U (pq = pair(mu <= nu)), then
//   E_M2^x = sum_{ijab} (ia|jb) [2 (ia|jb) - (ib|ja)] / (eps_i + eps_j - eps_a - eps_b).
// One block per fragment; workspace per fragment (global): A, V, C (n x n each), T1 [nocc][n][np],
// T2 [nocc][nvir][np], T3 [nocc][nvir][nocc][n], T4 [nocc][nvir][nocc][nvir].
__device__ __forceinline__ int m2_pair(int i, int j, int n)  // i <= j
{
    return i * n - i * (i - 1) / 2 + (j - i);
}

__global__ void __launch_bounds__(256) k_energy_m2(Dev d, const double* __restrict__ Fp, const double* __restrict__ Xp,
                                                   const int* __restrict__ nmo_, const double* __restrict__ Up,
                                                   const int64_t* __restrict__ ws_off, double* ws_all, double* E_out)
{
    const int x = blockIdx.x;
    const int n = d.frag_nao[x], m = nmo_[x], nocc = d.frag_nocc[x], nv = m - nocc;
    const int np = n * (n + 1) / 2;
    const Team<1> t{0};
    __shared__ JacobiScratch js;
    __shared__ double red[40];
    __shared__ int ord[kMaxFragAO];
    __shared__ double eps[kMaxFragAO];
    const int64_t mo = d.frag_moff[x];
    const double* F = Fp + mo;
    const double* X = Xp + mo;
    const double* U = Up + d.frag_coff[x];
    double* A = ws_all + ws_off[x];
    double* V = A + n * n;
    double* C = V + n * n;
    double* T1 = C + n * n;
    double* T2 = T1 + (int64_t)nocc * n * np;
    double* T3 = T2 + (int64_t)nocc * nv * np;
    double* T4 = T3 + (int64_t)nocc * nv * nocc * n;
    if (nocc <= 0 || nv <= 0) {
        if (threadIdx.x == 0) E_out[x] = 0.0;
        return;
    }
    mm(t, V, F, X, n, n, m, n, false);  // V = F X   (n x m)
    mm(t, A, X, V, m, n, m, n, true);   // A = X^T F X (m x m)
    jacobi_eigh(t, A, V, m, n, &js, red);
    if (threadIdx.x == 0) {  // ascending orbital energies, ties by index
        for (int k = 0; k < m; ++k) ord[k] = k;
        for (int k = 0; k < m; ++k) {
            int best = k;
            for (int j = k + 1; j < m; ++j) {
                const double ej = A[ord[j] * n + ord[j]], eb = A[ord[best] * n + ord[best]];
                if (ej < eb || (ej == eb && ord[j] < ord[best])) best = j;
            }
            const int tmp = ord[k]; ord[k] = ord[best]; ord[best] = tmp;
            eps[k] = A[ord[k] * n + ord[k]];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * m; e += blockDim.x) {  // C = X V, columns in ascending order
        const int mu = e / m, k = e % m;
        double sum = 0.0;
        for (int l = 0; l < m; ++l) sum = fma(X[mu * n + l], V[l * n + ord[k]], sum);
        C[mu * n + k] = sum;
    }
    __syncthreads();
    // T1[i][nu][rs] = sum_mu C[mu][i] U[pair(mu,nu)][rs]
    for (int64_t e = threadIdx.x; e < (int64_t)nocc * n * np; e += blockDim.x) {
        const int rs = (int)(e % np), nu = (int)((e / np) % n), i = (int)(e / ((int64_t)n * np));
        double sum = 0.0;
        for (int mu = 0; mu < n; ++mu)
            sum = fma(C[mu * n + i], U[(int64_t)(mu <= nu ? m2_pair(mu, nu, n) : m2_pair(nu, mu, n)) * np + rs], sum);
        T1[e] = sum;
    }
    __syncthreads();
    // T2[i][a][rs] = sum_nu C[nu][nocc + a] T1[i][nu][rs]
    for (int64_t e = threadIdx.x; e < (int64_t)nocc * nv * np; e += blockDim.x) {
        const int rs = (int)(e % np), a = (int)((e / np) % nv), i = (int)(e / ((int64_t)nv * np));
        double sum = 0.0;
        for (int nu = 0; nu < n; ++nu) sum = fma(C[nu * n + nocc + a], T1[((int64_t)i * n + nu) * np + rs], sum);
        T2[e] = sum;
    }
    __syncthreads();
    // T3[i][a][j][s] = sum_l C[l][j] T2[i][a][pair(l,s)]
    for (int64_t e = threadIdx.x; e < (int64_t)nocc * nv * nocc * n; e += blockDim.x) {
        const int sg = (int)(e % n), j = (int)((e / n) % nocc), ia = (int)(e / ((int64_t)nocc * n));
        double sum = 0.0;
        for (int l = 0; l < n; ++l)
            sum = fma(C[l * n + j], T2[(int64_t)ia * np + (l <= sg ? m2_pair(l, sg, n) : m2_pair(sg, l, n))], sum);
        T3[e] = sum;
    }
    __syncthreads();
    // T4[i][a][j][b] = sum_s C[s][nocc + b] T3[i][a][j][s]  (= (ia|jb))
    for (int64_t e = threadIdx.x; e < (int64_t)nocc * nv * nocc * nv; e += blockDim.x) {
        const int b = (int)(e % nv), iaj = (int)(e / nv);
        double sum = 0.0;
        for (int sg = 0; sg < n; ++sg) sum = fma(C[sg * n + nocc + b], T3[(int64_t)iaj * n + sg], sum);
        T4[e] = sum;
    }
    __syncthreads();
    double part = 0.0;
    for (int64_t e = threadIdx.x; e < (int64_t)nocc * nv * nocc * nv; e += blockDim.x) {
        const int b = (int)(e % nv), j = (int)((e / nv) % nocc), a = (int)((e / ((int64_t)nv * nocc)) % nv);
        const int i = (int)(e / ((int64_t)nv * nocc * nv));
        const double iajb = T4[e];
        const double ibja = T4[(((int64_t)i * nv + b) * nocc + j) * nv + a];
        part += iajb * (2.0 * iajb - ibja) / (eps[i] + eps[j] - eps[nocc + a] - eps[nocc + b]);
    }
    const double E = team_sum(t, part, red);
    if (threadIdx.x == 0) E_out[x] = E;
}

}  // namespace

int64_t energy_m2_workspace(int n, int nocc, int nmo)
{
    const int64_t np = (int64_t)n * (n + 1) / 2, nv = nmo - nocc;
    return 3 * (int64_t)n * n + (int64_t)nocc * n * np + nocc * nv * np + nocc * nv * nocc * n + nocc * nv * nocc * nv;
}

cudaError_t launch_energy_m2(const Dev& d, const double* F, const double* X, const int* nmo, const double* U,
                             const int64_t* ws_off, double* ws, double* E, cudaStream_t s)
{
    if (d.n_frag <= 0) return cudaSuccess;
    k_energy_m2<<<d.n_frag, 256, 0, s>>>(d, F, X, nmo, U, ws_off, ws, E);
    note_launches(1);
    return cudaGetLastError();
}

namespace {

// ------------------------------------------------------------------------------------------ E_D2
// Canonical FEF orbitals of every fragment (n <= kMaxFragAO): C (n x m, columns in ascending orbital
// energy) as the packed n x n block at frag_moff[x], eps[m] at frag_ao0[x]; one block per fragment,
// Jacobi workspace 2 n^2 at 2 frag_moff[x].
__global__ void __launch_bounds__(256) k_canonical_orbitals(Dev d, const double* __restrict__ Fp,
                                                            const double* __restrict__ Xp, const int* __restrict__ nmo_,
                                                            double* ws, double* Cp, double* eps_out)
{
    const int x = blockIdx.x;
    const int n = d.frag_nao[x], m = nmo_[x];
    const Team<1> t{0};
    __shared__ JacobiScratch js;
    __shared__ double red[40];
    __shared__ int ord[kMaxFragAO];
    const int64_t mo = d.frag_moff[x];
    const double* F = Fp + mo;
    const double* X = Xp + mo;
    double* A = ws + 2 * mo;
    double* V = A + n * n;
    double* C = Cp + mo;
    mm(t, V, F, X, n, n, m, n, false);
    mm(t, A, X, V, m, n, m, n, true);
    jacobi_eigh(t, A, V, m, n, &js, red);
    if (threadIdx.x == 0) {
        for (int k = 0; k < m; ++k) ord[k] = k;
        for (int k = 0; k < m; ++k) {
            int best = k;
            for (int j = k + 1; j < m; ++j) {
                const double ej = A[ord[j] * n + ord[j]], eb = A[ord[best] * n + ord[best]];
                if (ej < eb || (ej == eb && ord[j] < ord[best])) best = j;
            }
            const int tmp = ord[k]; ord[k] = ord[best]; ord[best] = tmp;
            eps_out[d.frag_ao0[x] + k] = A[ord[k] * n + ord[k]];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int mu = e / n, k = e % n;
        double sum = 0.0;
        if (k < m)
            for (int l = 0; l < m; ++l) sum = fma(X[mu * n + l], V[l * n + ord[k]], sum);
        C[e] = sum;
    }
}

// Dimer second-order term of one fragment pair (Eq. ED2 with the first-order dimer doubles of
// Eq. dimDoubles): one excitation on each fragment, direct interaction only (no inter-fragment
// exchange in the product ansatz), four spin cases:
//   E_D2^{xy} = 4 sum_{ia in x, jb in y} (ia|jb)^2 / (eps_i + eps_j - eps_a - eps_b),
// (ia|jb) by four quarter-transforms of the pair block W[pair(mu,nu) in x][pair(lambda,sigma) in y].
// One block per pair of the list; workspace per pair: T1 [nocc_x][n_x][np_y], T2 [nocc_x][nv_x][np_y],
// T3 [ov_x][nocc_y][n_y].
__global__ void __launch_bounds__(256) k_energy_d2(Dev d, const int* __restrict__ pair_of,
                                                   const int64_t* __restrict__ woff, const double* __restrict__ W,
                                                   const double* __restrict__ Cp, const double* __restrict__ eps,
                                                   const int* __restrict__ nmo_, const int64_t* __restrict__ toff,
                                                   double* tws, double* E_out)
{
    const int q = blockIdx.x;
    const int pr = pair_of[q];
    const int x = d.pair_x[pr], y = d.pair_y[pr];
    const int nx = d.frag_nao[x], ny = d.frag_nao[y];
    const int ox = d.frag_nocc[x], oy = d.frag_nocc[y];
    const int vx = nmo_[x] - ox, vy = nmo_[y] - oy;
    const int npy = ny * (ny + 1) / 2;
    const Team<1> t{0};
    __shared__ double red[40];
    const double* Wq = W + woff[q];
    const double* Cx = Cp + d.frag_moff[x];
    const double* Cy = Cp + d.frag_moff[y];
    const double* ex = eps + d.frag_ao0[x];
    const double* ey = eps + d.frag_ao0[y];
    double* T1 = tws + toff[q];
    double* T2 = T1 + (int64_t)ox * nx * npy;
    double* T3 = T2 + (int64_t)ox * vx * npy;
    for (int64_t e = threadIdx.x; e < (int64_t)ox * nx * npy; e += blockDim.x) {
        const int rs = (int)(e % npy), nu = (int)((e / npy) % nx), i = (int)(e / ((int64_t)nx * npy));
        double sum = 0.0;
        for (int mu = 0; mu < nx; ++mu) sum = fma(Cx[mu * nx + i], Wq[pair_pack(mu, nu, nx) * npy + rs], sum);
        T1[e] = sum;
    }
    __syncthreads();
    for (int64_t e = threadIdx.x; e < (int64_t)ox * vx * npy; e += blockDim.x) {
        const int rs = (int)(e % npy), a = (int)((e / npy) % vx), i = (int)(e / ((int64_t)vx * npy));
        double sum = 0.0;
        for (int nu = 0; nu < nx; ++nu) sum = fma(Cx[nu * nx + ox + a], T1[((int64_t)i * nx + nu) * npy + rs], sum);
        T2[e] = sum;
    }
    __syncthreads();
    for (int64_t e = threadIdx.x; e < (int64_t)ox * vx * oy * ny; e += blockDim.x) {
        const int sg = (int)(e % ny), j = (int)((e / ny) % oy), ia = (int)(e / ((int64_t)oy * ny));
        double sum = 0.0;
        for (int l = 0; l < ny; ++l) sum = fma(Cy[l * ny + j], T2[(int64_t)ia * npy + pair_pack(l, sg, ny)], sum);
        T3[e] = sum;
    }
    __syncthreads();
    double part = 0.0;
    for (int64_t e = threadIdx.x; e < (int64_t)ox * vx * oy * vy; e += blockDim.x) {
        const int b = (int)(e % vy), j = (int)((e / vy) % oy), a = (int)((e / ((int64_t)vy * oy)) % vx);
        const int i = (int)(e / ((int64_t)vy * oy * vx));
        const int64_t iaj = ((int64_t)i * vx + a) * oy + j;
        double v = 0.0;
        for (int sg = 0; sg < ny; ++sg) v = fma(Cy[sg * ny + oy + b], T3[iaj * ny + sg], v);
        part += v * v / (ex[i] + ey[j] - ex[ox + a] - ey[oy + b]);
    }
    const double E = team_sum(t, part, red);
    if (threadIdx.x == 0) E_out[q] = 4.0 * E;
}

}  // namespace

cudaError_t launch_canonical_orbitals(const Dev& d, const double* F, const double* X, const int* nmo, double* ws,
                                      double* C, double* eps, cudaStream_t s)
{
    if (d.n_frag <= 0) return cudaSuccess;
    k_canonical_orbitals<<<d.n_frag, 256, 0, s>>>(d, F, X, nmo, ws, C, eps);
    note_launches(1);
    return cudaGetLastError();
}

int64_t energy_d2_workspace(int nx, int ox, int mx, int ny, int oy, int my)
{
    const int64_t npy = (int64_t)ny * (ny + 1) / 2, vx = mx - ox, vy = my - oy;
    (void)vy;
    return (int64_t)ox * nx * npy + ox * vx * npy + ox * vx * oy * ny;
}

cudaError_t launch_energy_d2(const Dev& d, int n_pairs, const int* pair_of, const int64_t* woff, const double* W,
                             const double* C, const double* eps, const int* nmo, const int64_t* toff, double* tws,
                             double* E, cudaStream_t s)
{
    if (n_pairs <= 0) return cudaSuccess;
    k_energy_d2<<<n_pairs, 256, 0, s>>>(d, pair_of, woff, W, C, eps, nmo, toff, tws, E);
    note_launches(1);
    return cudaGetLastError();
}

namespace {
}  // namespace

// ------------------------------------------------------------------------------------------ X = U s^{-1/2}
// Also, when Sh / Sih are given: the symmetric square roots S^{1/2} = U s^{1/2} U^T and
// S^{-1/2} = U s^{-1/2} U^T (over s >= s_min), used to express densities in the Loewdin basis.
// Fragments above kOrthSmemMaxN AOs work in the global workspace ws (2 n^2 doubles at 2 frag_moff[x]).
__global__ void k_orthogonaliser(Dev d, const double* S, double* X, int* nmo_out, double s_min, double* Sh,
                                 double* Sih, double* ws)
{
    const int x = blockIdx.x;
    const int n = d.frag_nao[x];
    extern __shared__ double sm[];
    if (n > kOrthSmemMaxN && !ws) {
        if (threadIdx.x == 0) atomicOr(d.err_flag, kErrBounds);
        return;
    }
    double* A = n <= kOrthSmemMaxN ? sm : ws + 2 * d.frag_moff[x];
    double* V = A + n * n;
    __shared__ JacobiScratch js;
    __shared__ double red[40];
    __shared__ int keep_idx[kMaxFragAO];
    __shared__ int nkeep;
    const double* Sx = S + d.frag_moff[x];
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) A[e] = Sx[e];
    __syncthreads();
    jacobi_eigh(Team<1>{0}, A, V, n, n, &js, red);
    if (threadIdx.x == 0) {
        int c = 0;
        for (int k = 0; k < n; ++k)
            if (A[k * n + k] >= s_min) keep_idx[c++] = k;
        nkeep = c;
        nmo_out[x] = c;
    }
    __syncthreads();
    double* Xx = X + d.frag_moff[x];
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        int i = e / n, j = e % n;
        double v = 0.0;
        if (j < nkeep) {
            int k = keep_idx[j];
            v = V[i * n + k] * rsqrt(A[k * n + k]);
        }
        Xx[e] = v;
    }
    if (Sh || Sih) {
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            int i = e / n, j = e % n;
            double a = 0.0, b = 0.0;
            for (int k = 0; k < n; ++k) {
                double s = A[k * n + k];
                if (s < s_min) continue;
                double vv = V[i * n + k] * V[j * n + k];
                a += vv * sqrt(s);
                b += vv * rsqrt(s);
            }
            if (Sh) Sh[d.frag_moff[x] + e] = a;
            if (Sih) Sih[d.frag_moff[x] + e] = b;
        }
    }
}

cudaError_t launch_orthogonaliser(const Dev& d, const double* S, double* X, int* nmo, double s_min, int max_n,
                                  cudaStream_t s, double* Sh, double* Sih, double* ws)
{
    const size_t ns = (size_t)std::min(max_n, kOrthSmemMaxN);
    size_t smem = 2 * ns * ns * sizeof(double);
    cudaFuncSetAttribute(k_orthogonaliser, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_orthogonaliser<<<d.n_frag, 256, smem, s>>>(d, S, X, nmo, s_min, Sh, Sih, ws);
    note_launches(1);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------ fragment SCF
// PACKED: G from the packed transposed tensor CT[rs][pq] (setup.cu), thread per pq = (mu <= nu);
// otherwise from the full C[mu nu][lambda sigma], one warp per row.
// Working matrices Hw Ss Xs Ds Fs W A V Vp, nine n x n doubles (W doubles as the packed density):
// in shared memory up to kScfSmemMaxN AOs (one block per fragment, CS = 1), else in the global
// workspace a.ws at 9 frag_moff[x] (one thread-block cluster of CS blocks per fragment).
// The Jacobi of each micro-iteration starts from the previous eigenvectors Vp: A <- Vp^T A Vp,
// so only the small change of F' between iterations has to be rotated away.
template <bool PACKED, int CS>
__device__ __forceinline__ void fragment_scf(const Dev& d, const ScfArgs& a, const int x, const Team<CS> t,
                                             double* sm)
{
    const int n = d.frag_nao[x];
    const int m = a.nmo[x];
    const int nocc = d.frag_nocc[x];
    const int n2 = n * n;
    const int np = n * (n + 1) / 2;
    const int64_t mo = d.frag_moff[x];
    if ((CS == 1 && n > kScfSmemMaxN && !a.ws) || (CS > 1 && !a.ws)) {
        if (threadIdx.x == 0) atomicOr(d.err_flag, kErrBounds);
        return;
    }
    double* Hw = (CS == 1 && n <= kScfSmemMaxN) ? sm : a.ws + 9 * mo;
    double* Ss = Hw + n2;
    double* Xs = Ss + n2;
    double* Ds = Xs + n2;
    double* Fs = Ds + n2;
    double* W = Fs + n2;
    double* A = W + n2;
    double* V = A + n2;
    double* Vp = V + n2;
    __shared__ JacobiScratch js;
    __shared__ double red[40];
    __shared__ double B[8][8];
    __shared__ double coef[9];
    __shared__ int order[kMaxFragAO];
    __shared__ double gap;  // HOMO-LUMO gap of the last Roothaan step
    const int tid = threadIdx.x;
    if (tid == 0) gap = 0.0;
    const int g0 = t.g(), gs = t.gs();
    const int lane = tid & 31;
    const int gw = g0 >> 5, nw = gs >> 5;  // team-wide warp index and count
    const double* C = PACKED ? a.eric + d.frag_coff[x] : a.eric + d.frag_eoff[x];
    double* hF = a.diis_by_moff ? a.diis_F + 2 * (int64_t)a.diis_size * mo : a.diis_F + (int64_t)x * a.diis_stride;
    double* he = hF + (int64_t)a.diis_size * n2;

    for (int e = g0; e < n2; e += gs) {
        Hw[e] = a.h[mo + e] + (a.omega ? a.omega[mo + e] : 0.0);
        Ss[e] = a.S[mo + e];
        Xs[e] = a.X[mo + e];
        if (a.have_start) Ds[e] = a.D[mo + e];
    }
    t.sync();
    bool have_vp = false;
    double sigma = 0.0;         // level shift of the virtual orbitals: 0 until the fallback engages
    bool shift_density = false; // next shift relative to the occupied space of Ds (after a restart)

    // Roothaan step: W holds the (extrapolated) Fock matrix on entry; Ds gets the aufbau density.
    // With a level shift, sigma is added to the orbitals left empty by the previous step (in the
    // basis of the previous eigenvectors, where the previous occupation is diagonal): the shifted
    // matrix has the same eigenvectors at self-consistency, so only the path changes.
    auto roothaan = [&]() {
        mm(t, V, W, Xs, n, n, m, n, false);      // V = F X        (n x m)
        mm(t, A, Xs, V, m, n, m, n, true);       // A = X^T F X    (m x m)
        const double shift = (have_vp || shift_density) ? sigma : 0.0;
        if (!have_vp && shift != 0.0) {
            // A += shift (1 - P'), P' = (S X)^T D (S X) / 2 the occupied projector of Ds in the
            // orthonormal basis (W, V are free once A = X^T F X is formed)
            mm(t, V, Ss, Xs, n, n, m, n, false);  // V = S X      (n x m)
            mm(t, W, Ds, V, n, n, m, n, false);   // W = D S X    (n x m)
            for (int e = g0; e < m * m; e += gs) {
                const int i = e / m, j = e % m;
                double pij = 0.0;
                for (int l = 0; l < n; ++l) pij = fma(V[l * n + i], W[l * n + j], pij);
                A[i * n + j] += shift * ((i == j ? 1.0 : 0.0) - 0.5 * pij);
            }
            t.sync();
            shift_density = false;
        }
        if (have_vp) {
            mm(t, V, A, Vp, m, m, m, n, false);  // A <- Vp^T A Vp
            mm(t, A, Vp, V, m, m, m, n, true);
            if (shift != 0.0) {
                for (int j = g0; j < m; j += gs) {
                    bool occ = false;
                    for (int k = 0; k < nocc; ++k) occ = occ || order[k] == j;
                    if (!occ) A[j * n + j] += shift;
                }
                t.sync();
            }
        }
        jacobi_eigh(t, A, V, m, n, &js, red);    // A -> eigenvalues, V -> eigenvectors (m x m)
        if (have_vp) {
            mm(t, W, Vp, V, m, m, m, n, false);  // full eigenvectors Vp V
            for (int e = g0; e < m * m; e += gs) {
                int i = e / m, j = e % m;
                V[i * n + j] = W[i * n + j];
                Vp[i * n + j] = W[i * n + j];
            }
        } else {
            for (int e = g0; e < m * m; e += gs) {
                int i = e / m, j = e % m;
                Vp[i * n + j] = V[i * n + j];
            }
        }
        have_vp = true;
        t.sync();
        // ascending orbital energies, ties by index: thread k ranks eigenvalue k (every block of the
        // team orders the same eigenvalues the same way); the nocc lowest are occupied
        for (int k = tid; k < m; k += blockDim.x) {
            const double ek = A[k * n + k];
            int r = 0;
            for (int j = 0; j < m; ++j) {
                const double ej = A[j * n + j];
                r += (ej < ek || (ej == ek && j < k)) ? 1 : 0;
            }
            order[r] = k;
        }
        __syncthreads();
        if (tid == 0) {
            const double homo = nocc > 0 ? A[order[nocc - 1] * n + order[nocc - 1]] : 0.0;
            const double lumo = nocc < m ? A[order[nocc] * n + order[nocc]] : 0.0;
            gap = (nocc > 0 && nocc < m) ? lumo - homo - shift : 0.0;
        }
        for (int e = g0; e < n * nocc; e += gs) {  // W = C_occ = X V_occ  (n x nocc)
            int i = e / nocc, k = e % nocc;
            int col = order[k];
            double s = 0.0;
            for (int l = 0; l < m; ++l) s = fma(Xs[i * n + l], V[l * n + col], s);
            W[i * n + k] = s;
        }
        t.sync();
        for (int e = g0; e < n2; e += gs) {      // D = 2 C_occ C_occ^T
            int i = e / n, j = e % n;
            double s = 0.0;
            for (int k = 0; k < nocc; ++k) s = fma(W[i * n + k], W[j * n + k], s);
            Ds[e] = 2.0 * s;
        }
        t.sync();
    };

    if (!a.have_start) {  // core guess: F = h + omega
        for (int e = g0; e < n2; e += gs) W[e] = Hw[e];
        t.sync();
        roothaan();
    }

    double E_old = 0.0, E = 0.0;
    bool conv = false;
    int it = 0, it0 = 1;  // it0: first iteration of the current DIIS history
    // convergence thresholds: from device memory when given (set between graph replays)
    const double e_tol = a.tol ? a.tol[0] : a.e_tol;
    const double comm_tol = a.tol ? a.tol[1] : a.comm_tol;
    for (it = 1; it <= a.max_iter; ++it) {
        // fallback for a fragment that DIIS has not converged in shift_after iterations (DIIS can
        // wander where no aufbau solution lies): restart from the start density (or core guess)
        // with the virtual orbitals level-shifted and a fresh DIIS history
        if (a.shift_after > 0 && it == a.shift_after + 1) {
            sigma = a.level_shift;
            it0 = it;
            have_vp = false;
            if (a.have_start) {
                for (int e = g0; e < n2; e += gs) Ds[e] = a.D[mo + e];
                shift_density = true;
                t.sync();
            } else {
                for (int e = g0; e < n2; e += gs) W[e] = Hw[e];
                t.sync();
                roothaan();
            }
        }
        // F = h + omega + G[D]
        if (PACKED) {
            double* dpk = W;
            for (int rs = g0; rs < np; rs += gs) {
                int la = 0, r = rs;
                while (r >= n - la) { r -= n - la; ++la; }
                dpk[rs] = Ds[la * n + la + r];
            }
            t.sync();
            for (int pq = g0; pq < np; pq += gs) {
                int mu = 0, r = pq;
                while (r >= n - mu) { r -= n - mu; ++mu; }
                int nu = mu + r;
                double g = 0.0;
                for (int rs = 0; rs < np; ++rs) g = fma(C[(size_t)rs * np + pq], dpk[rs], g);
                Fs[mu * n + nu] = Hw[mu * n + nu] + g;
                Fs[nu * n + mu] = Hw[nu * n + mu] + g;
            }
        } else {
            for (int row = gw; row < n2; row += nw) {
                double g = 0.0;
                for (int c = lane; c < n2; c += 32) g = fma(C[(size_t)row * n2 + c], Ds[c], g);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
                if (lane == 0) Fs[row] = Hw[row] + g;
            }
        }
        t.sync();
        double part = 0.0;
        for (int e = g0; e < n2; e += gs) part += Ds[e] * (Hw[e] + Fs[e]);
        E = 0.5 * team_sum(t, part, red) + a.e_nn[x];
        // e = F D S - S D F = M - M^T with M = F D S
        mm(t, W, Fs, Ds, n, n, n, n, false);
        mm(t, V, W, Ss, n, n, n, n, false);
        double em = 0.0;
        for (int e = g0; e < n2; e += gs) {
            int i = e / n, j = e % n;
            em = fmax(em, fabs(V[i * n + j] - V[j * n + i]));
        }
        em = team_max(t, em, red);
        if (it > 1 && fabs(E - E_old) < e_tol && em < comm_tol) {
            conv = true;
            break;
        }
        if (!isfinite(E)) break;
        E_old = E;
        for (int e = g0; e < n2; e += gs) {
            int i = e / n, j = e % n;
            W[e] = V[i * n + j] - V[j * n + i];
        }
        t.sync();
        // DIIS history (ring of diis_size): F and X^T e X
        const int slot = (it - it0) % a.diis_size;
        const int hist = min(it - it0 + 1, a.diis_size);
        mm(t, V, W, Xs, n, n, m, n, false);  // V = e X
        mm(t, A, Xs, V, m, n, m, n, true);   // A = X^T e X
        for (int e = g0; e < n2; e += gs) {
            hF[(int64_t)slot * n2 + e] = Fs[e];
            int i = e / n, j = e % n;
            he[(int64_t)slot * n2 + e] = (i < m && j < m) ? A[i * n + j] : 0.0;
        }
        t.sync();
        // the new row of B: all hist dot products in one pass and one reduction per block (CS = 1);
        // across a cluster, one team reduction per product
        if constexpr (CS == 1) {
            double pj[8] = {};
            for (int e = g0; e < n2; e += gs) {
                const double se = he[(int64_t)slot * n2 + e];
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (j < hist) pj[j] = fma(se, he[(int64_t)j * n2 + e], pj[j]);
            }
            __shared__ double redh[8][8];
            const int w8 = tid >> 5;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                double v = pj[j];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0 && w8 < 8) redh[w8][j] = v;
            }
            __syncthreads();
            if (tid < hist) {
                double v = 0.0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += redh[w][tid];
                B[slot][tid] = v;
                B[tid][slot] = v;
            }
        } else {
            for (int j = 0; j < hist; ++j) {
                double pj = 0.0;
                for (int e = g0; e < n2; e += gs) pj += he[(int64_t)slot * n2 + e] * he[(int64_t)j * n2 + e];
                pj = team_sum(t, pj, red);
                if (tid == 0) {
                    B[slot][j] = pj;
                    B[j][slot] = pj;
                }
            }
        }
        __syncthreads();
        if (hist >= 2) {
            if (tid == 0) {  // solve [B -1; -1 0] [c; l] = [0; -1] by Gauss-Jordan, partial pivoting
                double M[9][10];
                const int sz = hist + 1;
                for (int i = 0; i < sz; ++i)
                    for (int j = 0; j <= sz; ++j) M[i][j] = 0.0;
                for (int i = 0; i < hist; ++i) {
                    for (int j = 0; j < hist; ++j) M[i][j] = B[i][j];
                    M[i][hist] = -1.0;
                    M[hist][i] = -1.0;
                }
                M[hist][sz] = -1.0;
                bool ok = true;
                for (int col = 0; col < sz; ++col) {
                    int piv = col;
                    for (int r = col + 1; r < sz; ++r)
                        if (fabs(M[r][col]) > fabs(M[piv][col])) piv = r;
                    if (fabs(M[piv][col]) < 1e-300) { ok = false; break; }
                    for (int j = 0; j <= sz; ++j) { double tmp = M[col][j]; M[col][j] = M[piv][j]; M[piv][j] = tmp; }
                    const double inv = 1.0 / M[col][col];  // one division per pivot
                    for (int r = 0; r < sz; ++r) {
                        if (r == col) continue;
                        const double f = M[r][col] * inv;
                        for (int j = col; j <= sz; ++j) M[r][j] -= f * M[col][j];
                    }
                }
                for (int i = 0; i < hist; ++i) coef[i] = ok ? M[i][sz] / M[i][i] : (i == slot ? 1.0 : 0.0);
            }
            __syncthreads();
            for (int e = g0; e < n2; e += gs) {
                double f = 0.0;
                for (int j = 0; j < hist; ++j) f = fma(coef[j], hF[(int64_t)j * n2 + e], f);
                W[e] = f;
            }
        } else {
            for (int e = g0; e < n2; e += gs) W[e] = Fs[e];
        }
        t.sync();
        roothaan();
    }
    // outputs: D and F of the returned density, energies
    double part = 0.0;
    for (int e = g0; e < n2; e += gs) {
        a.D[mo + e] = Ds[e];
        a.F[mo + e] = Fs[e];
        part += Ds[e] * (a.omega ? a.omega[mo + e] : 0.0);
    }
    double trw = team_sum(t, part, red);
    if (tid == 0 && t.rank == 0) {
        if (a.gap) a.gap[x] = gap;
        a.E_scf[x] = E;
        a.E_int[x] = E - trw;
        a.iters[x] = conv ? it : -a.max_iter;
        if (!conv) atomicOr(d.err_flag, isfinite(E) ? kErrNotConv : kErrNumeric);
    }
}

// One block per fragment (fragments a.list[0..n_list), or all when a.list is null).
template <bool PACKED>
__global__ void __launch_bounds__(256) k_fragment_scf(Dev d, ScfArgs a)
{
    extern __shared__ double sm[];
    const int x = a.list ? a.list[blockIdx.x] : (int)blockIdx.x;
    fragment_scf<PACKED, 1>(d, a, x, Team<1>{0}, sm);
}

// One cluster of CS blocks per fragment of a.big_list (matrices in the global workspace).
template <int CS>
__global__ void __launch_bounds__(256) k_fragment_scf_cluster(Dev d, ScfArgs a)
{
    const int rank = (int)cg::this_cluster().block_rank();
    const int x = a.big_list[blockIdx.x / CS];
    fragment_scf<true, CS>(d, a, x, Team<CS>{rank}, nullptr);
}

template <int CS>
static cudaError_t launch_cluster_scf(const Dev& d, const ScfArgs& a, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.n_big * CS);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_fragment_scf_cluster<CS>, d, a);
}

// Blocks per cluster for the fragments above the shared-memory limit: 16 where the device can
// co-schedule a 16-block cluster of this kernel, else 8 (portable).
static int scf_cluster_size()
{
    static int cs = 0;
    if (cs) return cs;
    cs = 8;
    if (cudaFuncSetAttribute(k_fragment_scf_cluster<16>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
        cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(16);
        cfg.blockDim = dim3(256);
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 16;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, k_fragment_scf_cluster<16>, &cfg) == cudaSuccess && n > 0) cs = 16;
    }
    cudaGetLastError();
    return cs;
}

cudaError_t launch_fragment_scf(const Dev& d, const ScfArgs& a, int max_n, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    if (a.n_big > 0) {  // large fragments first: their clusters run alongside the small-fragment blocks
        if (!a.eric_packed || !a.ws) return cudaErrorInvalidValue;
        e = scf_cluster_size() == 16 ? launch_cluster_scf<16>(d, a, s) : launch_cluster_scf<8>(d, a, s);
        if (e != cudaSuccess) return e;
        note_launches(1);
    }
    const int n_small = a.list ? a.n_list : d.n_frag;
    if (n_small <= 0) return cudaGetLastError();
    const int ns_max = a.list ? std::min(max_n, kScfSmemMaxN) : max_n;
    const size_t ns = (size_t)std::min(ns_max, kScfSmemMaxN);
    size_t smem = 9 * ns * ns * sizeof(double);
    auto kern = a.eric_packed ? k_fragment_scf<true> : k_fragment_scf<false>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<n_small, 256, smem, s>>>(d, a);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace fef
