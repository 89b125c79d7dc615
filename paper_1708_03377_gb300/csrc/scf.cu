// Fragment RHF in a frozen environment field (paper, "Fragment Mean Field": each fragment's
// determinant satisfies the Hartree-Fock equation with F~ = h(1) + (2J - K) + omega_x; the
// fragment orbitals are orthonormal in the fragment's own overlap metric S^x).
//
// One thread block per fragment runs the whole micro-iteration loop on the device:
//   G = C D (C: Coulomb-minus-half-exchange tensor), F = h + omega + G,
//   E_scf = tr[D (h + omega + F)]/2 + E_nn, e = F D S - S D F,
//   Pulay DIIS on X^T e X, F' = X^T F X, cyclic Jacobi eigensolver, aufbau, D = 2 C_occ C_occ^T,
// until |dE_scf| < e_tol and max|e| < comm_tol.  X = U s^{-1/2} is the canonical orthogonaliser.
#include "common.cuh"
#include "internal.hpp"

namespace fef {

namespace {

__device__ inline double block_sum(double v, double* red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w];
    __syncthreads();
    return s;
}

__device__ inline double block_max(double v, double* red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s = fmax(s, red[w]);
    __syncthreads();
    return s;
}

// C[m x k] = op(A) B with A, B, C row-major in shared memory, leading dimension ld.
// transA: C = A^T B with A stored k x m.
__device__ inline void mm(double* C, const double* A, const double* B, int m, int k, int ncol, int ld, bool transA)
{
    for (int e = threadIdx.x; e < m * ncol; e += blockDim.x) {
        int i = e / ncol, j = e % ncol;
        double s = 0.0;
        if (transA)
            for (int l = 0; l < k; ++l) s = fma(A[l * ld + i], B[l * ld + j], s);
        else
            for (int l = 0; l < k; ++l) s = fma(A[i * ld + l], B[l * ld + j], s);
        C[i * ld + j] = s;
    }
    __syncthreads();
}

struct JacobiScratch {
    double c[kMaxFragAO / 2], s[kMaxFragAO / 2];
    int p[kMaxFragAO / 2], q[kMaxFragAO / 2];
};

// Cyclic Jacobi on the symmetric m x m matrix A (shared or global, leading dimension ld),
// m <= kMaxFragAO.
// Parallel ordering: round-robin pairing (circle method), m/2 disjoint rotations per round, each
// zeroing A_pq with t = sgn(theta)/(|theta| + sqrt(theta^2 + 1)), theta = (A_qq - A_pp)/(2 A_pq)
// (Golub & Van Loan, symmetric Schur decomposition).
// On exit diag(A) holds the eigenvalues and the columns of V the eigenvectors.  Stops when the
// off-diagonal Frobenius norm is below 1e-14 times the largest diagonal magnitude.
__device__ void jacobi_eigh(double* A, double* V, int m, int ld, JacobiScratch* js, double* red)
{
    // A built from matrix products is symmetric only to rounding; an orthogonal similarity keeps
    // the antisymmetric part, so symmetrise first and measure convergence on the upper triangle.
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        int r = e / m, c = e % m;
        V[r * ld + c] = (r == c) ? 1.0 : 0.0;
        if (r < c) {
            double v = 0.5 * (A[r * ld + c] + A[c * ld + r]);
            A[r * ld + c] = v;
            A[c * ld + r] = v;
        }
    }
    __syncthreads();
    const int M = m + (m & 1);
    const int half = M / 2;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, dg = 0.0;
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            int r = e / m, c = e % m;
            double v = A[r * ld + c];
            if (r < c) off += 2.0 * v * v; else if (r == c) dg = fmax(dg, fabs(v));
        }
        off = block_sum(off, red);
        dg = block_max(dg, red);
        if (off <= 1e-28 * fmax(dg * dg, 1e-300)) break;
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
                        float t = 1.0f / (fabsf(theta) + sqrtf(fmaf(theta, theta, 1.0f)));
                        if (theta < 0.0f) t = -t;
                        const double td = (double)t;
                        c = rsqrt(fma(td, td, 1.0));
                        s = td * c;
                    }
                }
                js->p[k] = p;
                js->q[k] = q;
                js->c[k] = c;
                js->s[k] = s;
            }
            __syncthreads();
            for (int w = threadIdx.x; w < half * m; w += blockDim.x) {
                int k = w / m, j = w % m;
                int p = js->p[k], q = js->q[k];
                if (q >= m || js->s[k] == 0.0) continue;
                double c = js->c[k], s = js->s[k];
                double ap = A[p * ld + j], aq = A[q * ld + j];
                A[p * ld + j] = c * ap - s * aq;
                A[q * ld + j] = s * ap + c * aq;
            }
            __syncthreads();
            for (int w = threadIdx.x; w < half * m; w += blockDim.x) {
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
            __syncthreads();
        }
    }
}

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
    __shared__ double red[32];
    __shared__ int keep_idx[kMaxFragAO];
    __shared__ int nkeep;
    const double* Sx = S + d.frag_moff[x];
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) A[e] = Sx[e];
    __syncthreads();
    jacobi_eigh(A, V, n, n, &js, red);
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
// in shared memory up to kScfSmemMaxN AOs, else in the global workspace a.ws at 9 frag_moff[x].
// The Jacobi of each micro-iteration starts from the previous eigenvectors Vp: A <- Vp^T A Vp,
// so only the small change of F' between iterations has to be rotated away.
template <bool PACKED>
__global__ void __launch_bounds__(256) k_fragment_scf(Dev d, ScfArgs a)
{
    const int x = blockIdx.x;
    const int n = d.frag_nao[x];
    const int m = a.nmo[x];
    const int nocc = d.frag_nocc[x];
    const int n2 = n * n;
    const int np = n * (n + 1) / 2;
    const int64_t mo = d.frag_moff[x];
    extern __shared__ double sm[];
    if (n > kScfSmemMaxN && !a.ws) {
        if (threadIdx.x == 0) atomicOr(d.err_flag, kErrBounds);
        return;
    }
    double* Hw = n <= kScfSmemMaxN ? sm : a.ws + 9 * mo;
    double* Ss = Hw + n2;
    double* Xs = Ss + n2;
    double* Ds = Xs + n2;
    double* Fs = Ds + n2;
    double* W = Fs + n2;
    double* A = W + n2;
    double* V = A + n2;
    double* Vp = V + n2;
    __shared__ JacobiScratch js;
    __shared__ double red[32];
    __shared__ double B[8][8];
    __shared__ double coef[9];
    __shared__ int order[kMaxFragAO];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const double* C = PACKED ? a.eric + d.frag_coff[x] : a.eric + d.frag_eoff[x];
    double* hF = a.diis_by_moff ? a.diis_F + 2 * (int64_t)a.diis_size * mo : a.diis_F + (int64_t)x * a.diis_stride;
    double* he = hF + (int64_t)a.diis_size * n2;

    for (int e = tid; e < n2; e += nt) {
        Hw[e] = a.h[mo + e] + (a.omega ? a.omega[mo + e] : 0.0);
        Ss[e] = a.S[mo + e];
        Xs[e] = a.X[mo + e];
        if (a.have_start) Ds[e] = a.D[mo + e];
    }
    __syncthreads();
    bool have_vp = false;

    // Roothaan step: W holds the (extrapolated) Fock matrix on entry; Ds gets the aufbau density.
    auto roothaan = [&]() {
        mm(V, W, Xs, n, n, m, n, false);      // V = F X        (n x m)
        mm(A, Xs, V, m, n, m, n, true);       // A = X^T F X    (m x m)
        if (have_vp) {
            mm(V, A, Vp, m, m, m, n, false);  // A <- Vp^T A Vp
            mm(A, Vp, V, m, m, m, n, true);
        }
        jacobi_eigh(A, V, m, n, &js, red);    // A -> eigenvalues, V -> eigenvectors (m x m)
        if (have_vp) {
            mm(W, Vp, V, m, m, m, n, false);  // full eigenvectors Vp V
            for (int e = tid; e < m * m; e += nt) {
                int i = e / m, j = e % m;
                V[i * n + j] = W[i * n + j];
                Vp[i * n + j] = W[i * n + j];
            }
        } else {
            for (int e = tid; e < m * m; e += nt) {
                int i = e / m, j = e % m;
                Vp[i * n + j] = V[i * n + j];
            }
        }
        have_vp = true;
        __syncthreads();
        if (tid == 0) {
            for (int k = 0; k < m; ++k) order[k] = k;
            for (int k = 0; k < nocc; ++k) {  // selection of the nocc lowest, ties by index
                int best = k;
                for (int j = k + 1; j < m; ++j) {
                    double ej = A[order[j] * n + order[j]], eb = A[order[best] * n + order[best]];
                    if (ej < eb || (ej == eb && order[j] < order[best])) best = j;
                }
                int t = order[k]; order[k] = order[best]; order[best] = t;
            }
        }
        __syncthreads();
        for (int e = tid; e < n * nocc; e += nt) {  // W = C_occ = X V_occ  (n x nocc)
            int i = e / nocc, k = e % nocc;
            int col = order[k];
            double s = 0.0;
            for (int l = 0; l < m; ++l) s = fma(Xs[i * n + l], V[l * n + col], s);
            W[i * n + k] = s;
        }
        __syncthreads();
        for (int e = tid; e < n2; e += nt) {      // D = 2 C_occ C_occ^T
            int i = e / n, j = e % n;
            double s = 0.0;
            for (int k = 0; k < nocc; ++k) s = fma(W[i * n + k], W[j * n + k], s);
            Ds[e] = 2.0 * s;
        }
        __syncthreads();
    };

    if (!a.have_start) {  // core guess: F = h + omega
        for (int e = tid; e < n2; e += nt) W[e] = Hw[e];
        __syncthreads();
        roothaan();
    }

    double E_old = 0.0, E = 0.0;
    bool conv = false;
    int it = 0;
    for (it = 1; it <= a.max_iter; ++it) {
        // F = h + omega + G[D]
        if (PACKED) {
            double* dpk = W;
            for (int rs = tid; rs < np; rs += nt) {
                int la = 0, r = rs;
                while (r >= n - la) { r -= n - la; ++la; }
                dpk[rs] = Ds[la * n + la + r];
            }
            __syncthreads();
            for (int pq = tid; pq < np; pq += nt) {
                int mu = 0, r = pq;
                while (r >= n - mu) { r -= n - mu; ++mu; }
                int nu = mu + r;
                double g = 0.0;
                for (int rs = 0; rs < np; ++rs) g = fma(C[(size_t)rs * np + pq], dpk[rs], g);
                Fs[mu * n + nu] = Hw[mu * n + nu] + g;
                Fs[nu * n + mu] = Hw[nu * n + mu] + g;
            }
        } else {
            for (int row = warp; row < n2; row += nw) {
                double g = 0.0;
                for (int c = lane; c < n2; c += 32) g = fma(C[(size_t)row * n2 + c], Ds[c], g);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
                if (lane == 0) Fs[row] = Hw[row] + g;
            }
        }
        __syncthreads();
        double part = 0.0;
        for (int e = tid; e < n2; e += nt) part += Ds[e] * (Hw[e] + Fs[e]);
        E = 0.5 * block_sum(part, red) + a.e_nn[x];
        // e = F D S - S D F = M - M^T with M = F D S
        mm(W, Fs, Ds, n, n, n, n, false);
        mm(V, W, Ss, n, n, n, n, false);
        double em = 0.0;
        for (int e = tid; e < n2; e += nt) {
            int i = e / n, j = e % n;
            em = fmax(em, fabs(V[i * n + j] - V[j * n + i]));
        }
        em = block_max(em, red);
        if (it > 1 && fabs(E - E_old) < a.e_tol && em < a.comm_tol) {
            conv = true;
            break;
        }
        if (!isfinite(E)) break;
        E_old = E;
        for (int e = tid; e < n2; e += nt) {
            int i = e / n, j = e % n;
            W[e] = V[i * n + j] - V[j * n + i];
        }
        __syncthreads();
        // DIIS history (ring of diis_size): F and X^T e X
        const int slot = (it - 1) % a.diis_size;
        const int hist = min(it, a.diis_size);
        mm(V, W, Xs, n, n, m, n, false);  // V = e X
        mm(A, Xs, V, m, n, m, n, true);   // A = X^T e X
        for (int e = tid; e < n2; e += nt) {
            hF[(int64_t)slot * n2 + e] = Fs[e];
            int i = e / n, j = e % n;
            he[(int64_t)slot * n2 + e] = (i < m && j < m) ? A[i * n + j] : 0.0;
        }
        __syncthreads();
        for (int j = 0; j < hist; ++j) {
            double p = 0.0;
            for (int e = tid; e < n2; e += nt) p += he[(int64_t)slot * n2 + e] * he[(int64_t)j * n2 + e];
            p = block_sum(p, red);
            if (tid == 0) {
                B[slot][j] = p;
                B[j][slot] = p;
            }
        }
        __syncthreads();
        if (hist >= 2) {
            if (tid == 0) {  // solve [B -1; -1 0] [c; l] = [0; -1] by Gauss-Jordan, partial pivoting
                double M[9][10];
                const int s = hist + 1;
                for (int i = 0; i < s; ++i)
                    for (int j = 0; j <= s; ++j) M[i][j] = 0.0;
                for (int i = 0; i < hist; ++i) {
                    for (int j = 0; j < hist; ++j) M[i][j] = B[i][j];
                    M[i][hist] = -1.0;
                    M[hist][i] = -1.0;
                }
                M[hist][s] = -1.0;
                bool ok = true;
                for (int col = 0; col < s; ++col) {
                    int piv = col;
                    for (int r = col + 1; r < s; ++r)
                        if (fabs(M[r][col]) > fabs(M[piv][col])) piv = r;
                    if (fabs(M[piv][col]) < 1e-300) { ok = false; break; }
                    for (int j = 0; j <= s; ++j) { double t = M[col][j]; M[col][j] = M[piv][j]; M[piv][j] = t; }
                    for (int r = 0; r < s; ++r) {
                        if (r == col) continue;
                        double f = M[r][col] / M[col][col];
                        for (int j = col; j <= s; ++j) M[r][j] -= f * M[col][j];
                    }
                }
                for (int i = 0; i < hist; ++i) coef[i] = ok ? M[i][s] / M[i][i] : (i == slot ? 1.0 : 0.0);
            }
            __syncthreads();
            for (int e = tid; e < n2; e += nt) {
                double f = 0.0;
                for (int j = 0; j < hist; ++j) f = fma(coef[j], hF[(int64_t)j * n2 + e], f);
                W[e] = f;
            }
        } else {
            for (int e = tid; e < n2; e += nt) W[e] = Fs[e];
        }
        __syncthreads();
        roothaan();
    }
    // outputs: D and F of the returned density, energies
    double part = 0.0;
    for (int e = tid; e < n2; e += nt) {
        a.D[mo + e] = Ds[e];
        a.F[mo + e] = Fs[e];
        part += Ds[e] * (a.omega ? a.omega[mo + e] : 0.0);
    }
    double trw = block_sum(part, red);
    if (tid == 0) {
        a.E_scf[x] = E;
        a.E_int[x] = E - trw;
        a.iters[x] = conv ? it : -a.max_iter;
        if (!conv) atomicOr(d.err_flag, isfinite(E) ? kErrNotConv : kErrNumeric);
    }
}

cudaError_t launch_fragment_scf(const Dev& d, const ScfArgs& a, int max_n, cudaStream_t s)
{
    const size_t ns = (size_t)std::min(max_n, kScfSmemMaxN);
    size_t smem = 9 * ns * ns * sizeof(double);
    auto kern = a.eric_packed ? k_fragment_scf<true> : k_fragment_scf<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<d.n_frag, 256, smem, s>>>(d, a);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace fef
