// Inputs and outputs of the learned warm start, in each fragment's molecule-fixed frame.
//
// Frame of fragment x: e1 along R_1 - R_0, e2 the part of R_2 - R_0 orthogonal to e1, e3 = e1 x e2
// (atoms in input order); the rotation Rot has these axes as columns, r_global = Rot r_local.
// Descriptors: at every atom A of x, the electrostatic potential and field of all neighbour
// fragments y in N(x) (their nuclei and their electron densities D^y), the field rotated into the
// frame:   phi(A) = sum_{B in y} Z_B/|A-B| - sum_Q sum_tuv Dt_Q[tuv] (2 pi/q) R_tuv(q, Q - A),
//          E(A)   = sum_{B in y} Z_B (A-B)/|A-B|^3 - sum_Q sum_tuv Dt_Q[tuv] (2 pi/q) R_{t+e}(q, Q - A),
// with Dt_Q the Hermite density of primitive pair Q (McMurchie-Davidson, as in the J-engine).
// Densities in the frame and in the Loewdin basis: with B the AO transformation of the frame (1 for
// s, Rot for p; orthogonal), D_local = B^T S^{1/2} D S^{1/2} B and back D = S^{-1/2} B D_local B^T
// S^{-1/2}.  The Loewdin basis keeps the learned quantity well conditioned: in the AO basis a
// density change is dominated by near-linearly-dependent directions of S.
#include "common.cuh"
#include "internal.hpp"

namespace fef {

__global__ void k_frames(Dev d, double* rot)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= d.n_frag) return;
    const int a0 = d.frag_atom0[x], nat = d.frag_nat[x];
    double e1[3] = {1, 0, 0}, e2[3] = {0, 1, 0}, e3[3] = {0, 0, 1};
    if (nat >= 2) {
        const double* A = d.atom_xyz + 3 * a0;
        const double* B = d.atom_xyz + 3 * (a0 + 1);
        double n = 0;
        for (int k = 0; k < 3; ++k) { e1[k] = B[k] - A[k]; n += e1[k] * e1[k]; }
        n = sqrt(n);
        for (int k = 0; k < 3; ++k) e1[k] /= n;
        double v[3];
        if (nat >= 3) {
            const double* C = d.atom_xyz + 3 * (a0 + 2);
            for (int k = 0; k < 3; ++k) v[k] = C[k] - A[k];
        } else {
            v[0] = fabs(e1[0]) < 0.9 ? 1.0 : 0.0;
            v[1] = fabs(e1[0]) < 0.9 ? 0.0 : 1.0;
            v[2] = 0.0;
        }
        double dot = v[0] * e1[0] + v[1] * e1[1] + v[2] * e1[2];
        n = 0;
        for (int k = 0; k < 3; ++k) { e2[k] = v[k] - dot * e1[k]; n += e2[k] * e2[k]; }
        n = sqrt(n);
        for (int k = 0; k < 3; ++k) e2[k] /= n;
        e3[0] = e1[1] * e2[2] - e1[2] * e2[1];
        e3[1] = e1[2] * e2[0] - e1[0] * e2[2];
        e3[2] = e1[0] * e2[1] - e1[1] * e2[0];
    }
    double* R = rot + 9 * x;  // row-major, columns = local axes
    for (int k = 0; k < 3; ++k) {
        R[3 * k + 0] = e1[k];
        R[3 * k + 1] = e2[k];
        R[3 * k + 2] = e3[k];
    }
}

// Potential and field at the point r (relative to the anchor of the pair's fragment) from the
// Hermite density Dt of one primitive pair of class L with centre Pr (same anchor) and exponent p,
// all in FP32 (the descriptors are FP32 network inputs): Boys, R recursion and contraction.
template <int L>
__device__ __forceinline__ void pair_potential32(const float* __restrict__ boys32, float4 Pr, const float* Dt,
                                                 const float* r, float* out)
{
    const float q = Pr.w;
    const float X = Pr.x - r[0], Y = Pr.y - r[1], Z = Pr.z - r[2];
    float F[L + 2], base[L + 2], R[nh(L + 1)];
    boys_fp32<L + 1>(boys32, q * (X * X + Y * Y + Z * Z), F);
    float f = 2.0f * (float)kPi / q;
#pragma unroll
    for (int n = 0; n <= L + 1; ++n) {
        base[n] = f * F[n];
        f *= -2.0f * q;
    }
    md_R<L + 1, float>(R, base, X, Y, Z);
    static_for<nh(L)>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        constexpr TUV c = htuv(k);
        out[0] = fmaf(-Dt[k], R[k], out[0]);
        out[1] = fmaf(-Dt[k], R[hidx(c.t + 1, c.u, c.v)], out[1]);
        out[2] = fmaf(-Dt[k], R[hidx(c.t, c.u + 1, c.v)], out[2]);
        out[3] = fmaf(-Dt[k], R[hidx(c.t, c.u, c.v + 1)], out[3]);
    });
}

// FP32 Hermite densities of the current densities for the descriptors, Dt = Dh p / (2 pi^{5/2})
// (Dh holds D K c 2 pi^{5/2} / p), into the FP32 scratch pp_Dh32.
__global__ void k_descriptor_density(Dev d, int L)
{
    const int npp = d.n_pp[L];
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= npp) return;
    const double sc = d.pp_P[L][g].w * (1.0 / kSqrt2Pi52);
    for (int k = 0; k < nh(L); ++k) d.pp_Dh32[L][(size_t)k * npp + g] = (float)(d.pp_Dh[L][(size_t)k * npp + g] * sc);
}

// Descriptors in two steps.  k_descriptor_terms: one block per neighbour entry c = (x, y) of the CSR
// list; its threads split y's nuclei and primitive pairs, each item contributes to every atom of x
// (atoms and pair centres relative to y's anchor atom, FP32 terms and per-thread sums), and the block
// writes its sums (phi, E) per atom to part[(c max_nat + a) 4 ..] (FP64 block reduction).
// k_descriptor_sum: one thread per (x, a) adds its neighbours' parts in list order (reproducible) and
// writes X[x][4a + (0..3)] = (phi, E in the frame).
constexpr int kDescThreads = 128;
constexpr int kDescAtoms = 4;  // atoms of x per pass over y's items

__global__ void __launch_bounds__(kDescThreads) k_descriptor_terms(Dev d, int max_nat, double* part)
{
    __shared__ double red[kDescThreads / 32][kDescAtoms * 4];
    __shared__ float rel[kDescAtoms][3];
    const int c = blockIdx.x;
    int lo = 0, hi = d.n_frag - 1;  // fragment x owning entry c (frag_nbr0 ascending)
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (d.frag_nbr0[mid] <= c) lo = mid; else hi = mid - 1;
    }
    const int x = lo, y = d.nbr[c];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nat = d.frag_nat[x], naty = d.frag_nat[y];
    const double* anc = d.atom_xyz + 3 * d.frag_atom0[y];
    for (int a0 = 0; a0 < max_nat; a0 += kDescAtoms) {
        const int na = max(0, min(kDescAtoms, nat - a0));
        if (tid < 3 * kDescAtoms) {
            const int a = tid / 3, k = tid % 3;
            rel[a][k] = a < na ? (float)(d.atom_xyz[3 * (d.frag_atom0[x] + a0 + a) + k] - anc[k]) : 0.0f;
        }
        __syncthreads();
        float v[kDescAtoms][4] = {};
        // nuclei of y
        for (int t = tid; t < naty; t += kDescThreads) {
            const float Zb = (float)d.atom_Z[d.frag_atom0[y] + t];
            const float bx = (float)(d.atom_xyz[3 * (d.frag_atom0[y] + t)] - anc[0]);
            const float by = (float)(d.atom_xyz[3 * (d.frag_atom0[y] + t) + 1] - anc[1]);
            const float bz = (float)(d.atom_xyz[3 * (d.frag_atom0[y] + t) + 2] - anc[2]);
#pragma unroll
            for (int a = 0; a < kDescAtoms; ++a) {
                if (a >= na) break;
                const float dx = rel[a][0] - bx, dy = rel[a][1] - by, dz = rel[a][2] - bz;
                const float ir = rsqrtf(dx * dx + dy * dy + dz * dz);
                const float f = Zb * ir * ir * ir;
                v[a][0] += Zb * ir;
                v[a][1] += f * dx;
                v[a][2] += f * dy;
                v[a][3] += f * dz;
            }
        }
        // primitive pairs of y, class by class (s/p fragments: L <= 2)
#pragma unroll
        for (int L = 0; L <= 2; ++L) {
            const int g0 = d.frag_pp0[y * kClasses + L], ng = d.frag_npp[y * kClasses + L];
            const int npp = d.n_pp[L];
            for (int u = tid; u < ng; u += kDescThreads) {
                const int g = g0 + u;
                const float4 Pr = d.pp_Pr[L][g];
                float Dt[nh(2)];
                for (int k = 0; k < nh(L); ++k) Dt[k] = d.pp_Dh32[L][(size_t)k * npp + g];
#pragma unroll
                for (int a = 0; a < kDescAtoms; ++a) {
                    if (a >= na) break;
                    if (L == 0) pair_potential32<0>(d.boys32, Pr, Dt, rel[a], v[a]);
                    else if (L == 1) pair_potential32<1>(d.boys32, Pr, Dt, rel[a], v[a]);
                    else pair_potential32<2>(d.boys32, Pr, Dt, rel[a], v[a]);
                }
            }
        }
#pragma unroll
        for (int a = 0; a < kDescAtoms; ++a)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                double w = (double)v[a][k];
                for (int off = 16; off > 0; off >>= 1) w += __shfl_xor_sync(0xffffffffu, w, off);
                if (lane == 0) red[warp][4 * a + k] = w;
            }
        __syncthreads();
        if (tid < 4 * na) {
            double s4 = 0.0;
            for (int w = 0; w < kDescThreads / 32; ++w) s4 += red[w][tid];
            part[((size_t)c * max_nat + a0 + tid / 4) * 4 + tid % 4] = s4;
        }
        __syncthreads();
    }
}

__global__ void k_descriptor_sum(Dev d, const double* rot, int n_feat, int max_nat, const double* __restrict__ part,
                                 float* X)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n_frag * max_nat) return;
    const int x = i / max_nat, a = i % max_nat;
    if (a >= d.frag_nat[x]) return;
    double s4[4] = {0.0, 0.0, 0.0, 0.0};
    for (int c = d.frag_nbr0[x]; c < d.frag_nbr0[x + 1]; ++c)
        for (int k = 0; k < 4; ++k) s4[k] += part[((size_t)c * max_nat + a) * 4 + k];
    const double* R = rot + 9 * x;
    float* out = X + (size_t)x * n_feat + 4 * a;
    out[0] = (float)s4[0];
    for (int k = 0; k < 3; ++k) out[1 + k] = (float)(R[0 * 3 + k] * s4[1] + R[1 * 3 + k] * s4[2] + R[2 * 3 + k] * s4[3]);
}

// B (n x n) of fragment x into shared memory: 1 on s functions, Rot on each p shell.
__device__ inline void frame_ao_matrix(const Dev& d, int x, const double* Rt, double* B, int n)
{
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) B[e] = 0.0;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int s = d.frag_sh0[x]; s < d.frag_sh0[x] + d.frag_nsh[x]; ++s) {
            const int o = d.sh_ao[s];
            if (d.sh_l[s] == 0) {
                B[o * n + o] = 1.0;
            } else {  // p (d shells are rejected by the caller)
                for (int k = 0; k < 3; ++k)
                    for (int m = 0; m < 3; ++m) B[(o + k) * n + o + m] = Rt[3 * k + m];
            }
        }
    }
    __syncthreads();
}

// out[x][packed i<=j] = (B^T S^{1/2} D S^{1/2} B)_ij, one block per fragment.  Passing S^{-1/2} as Sh
// gives the Loewdin-basis form of an operator instead (S^{-1/2} F S^{-1/2}), so that tr(D F) is kept.
// out row stride is `stride` floats, written from column `col0`.
__global__ void k_local_density(Dev d, const double* rot, const double* Sh, const double* D, int stride, int col0,
                                float* out)
{
    const int x = blockIdx.x;
    const int n = d.frag_nao[x];
    extern __shared__ double sm[];
    double* B = sm;
    double* T = B + n * n;
    double* U = T + n * n;
    frame_ao_matrix(d, x, rot + 9 * x, B, n);
    const double* Dx = D + d.frag_moff[x];
    const double* Hx = Sh + d.frag_moff[x];
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {  // T = D S^{1/2}
        int i = e / n, j = e % n;
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += Dx[i * n + k] * Hx[k * n + j];
        T[e] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {  // U = S^{1/2} T
        int i = e / n, j = e % n;
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += Hx[i * n + k] * T[k * n + j];
        U[e] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {  // T = U B
        int i = e / n, j = e % n;
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += U[i * n + k] * B[k * n + j];
        T[e] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * (n + 1) / 2; e += blockDim.x) {  // (B^T T)_ij, i <= j
        int i = 0, r = e;
        while (r >= n - i) { r -= n - i; ++i; }
        int j = i + r;
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += B[k * n + i] * T[k * n + j];
        out[(size_t)x * stride + col0 + e] = (float)s;
    }
}

// D = D_iso + S^{-1/2} B dL B^T S^{-1/2} with dL the packed local-frame Loewdin-basis density
// change; one block per fragment.
__global__ void k_apply_learned(Dev d, const double* rot, const double* Sih, const double* D_iso, const float* dloc,
                                int n_pack, double* D)
{
    const int x = blockIdx.x;
    const int n = d.frag_nao[x];
    extern __shared__ double sm[];
    double* B = sm;
    double* M = B + n * n;
    double* T = M + n * n;
    frame_ao_matrix(d, x, rot + 9 * x, B, n);
    const double* Gx = Sih + d.frag_moff[x];
    for (int e = threadIdx.x; e < n * (n + 1) / 2; e += blockDim.x) {
        int i = 0, r = e;
        while (r >= n - i) { r -= n - i; ++i; }
        int j = i + r;
        double v = (double)dloc[(size_t)x * n_pack + e];
        M[i * n + j] = v;
        M[j * n + i] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {  // T = M B^T
        int i = e / n, j = e % n;
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += M[i * n + k] * B[j * n + k];
        T[e] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {  // M = B T  (global-frame Loewdin change)
        int i = e / n, j = e % n;
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += B[i * n + k] * T[k * n + j];
        M[e] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {  // T = M S^{-1/2}
        int i = e / n, j = e % n;
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += M[i * n + k] * Gx[k * n + j];
        T[e] = s;
    }
    __syncthreads();
    const int64_t mo = d.frag_moff[x];
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {  // D = D_iso + S^{-1/2} T
        int i = e / n, j = e % n;
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += Gx[i * n + k] * T[k * n + j];
        D[mo + e] = D_iso[mo + e] + s;
    }
}

cudaError_t launch_frames(const Dev& d, double* rot, cudaStream_t s)
{
    k_frames<<<(d.n_frag + 127) / 128, 128, 0, s>>>(d, rot);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_descriptors(const Dev& d, const double* rot, int n_feat, int max_nat, int n_nbr, double* part,
                               float* X, cudaStream_t s)
{
    if (d.n_frag <= 0) return cudaSuccess;
    if (n_nbr > 0) {
        for (int L = 0; L <= 2; ++L)
            if (d.n_pp[L] > 0) {
                k_descriptor_density<<<(d.n_pp[L] + 127) / 128, 128, 0, s>>>(d, L);
                note_launches(1);
            }
        k_descriptor_terms<<<(unsigned)n_nbr, kDescThreads, 0, s>>>(d, max_nat, part);
        note_launches(1);
    }
    k_descriptor_sum<<<(d.n_frag * max_nat + 127) / 128, 128, 0, s>>>(d, rot, n_feat, max_nat, part, X);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_local_density(const Dev& d, const double* rot, const double* Sh, const double* D, int stride,
                                 int col0, float* out, cudaStream_t s)
{
    size_t smem = 3 * sizeof(double) * (size_t)d.max_nao * d.max_nao;
    cudaFuncSetAttribute(k_local_density, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_local_density<<<d.n_frag, 128, smem, s>>>(d, rot, Sh, D, stride, col0, out);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_apply_learned(const Dev& d, const double* rot, const double* Sih, const double* D_iso,
                                 const float* dloc, int n_pack, double* D, cudaStream_t s)
{
    size_t smem = 3 * sizeof(double) * (size_t)d.max_nao * d.max_nao;
    cudaFuncSetAttribute(k_apply_learned, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_apply_learned<<<d.n_frag, 128, smem, s>>>(d, rot, Sih, D_iso, dloc, n_pack, D);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace fef
