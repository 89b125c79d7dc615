// Device building blocks of the FEF effective-field Fock build on sm_103a.
//
// Integrals follow McMurchie & Davidson (J. Comput. Phys. 26, 218 (1978)): a product of two
// Cartesian Gaussians is expanded in Hermite Gaussians with coefficients E^{ij}_t, and every
// Coulomb-type integral reduces to the Hermite integrals R_{tuv}(alpha, PQ) built from the Boys
// function F_n(T) = int_0^1 t^{2n} exp(-T t^2) dt.  These integrals realise the one-electron part
// h(1), the inter-fragment nuclear attraction h~ and the two-electron integrals of Eq. dp2e of the
// paper's "Fragment Mean Field" section.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

namespace fef {

// Compile-time loop: f(std::integral_constant<int, i>) for i = 0..N-1, so that array indices
// derived from i are constants and the arrays stay in registers.
template <typename F, int... I>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, I...>)
{
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void static_for(F&& f)
{
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

constexpr double kPi = 3.14159265358979323846;
// sqrt(2 pi^{5/2}): split evenly between bra and ket Hermite densities so that the per-quartet
// prefactor 2 pi^{5/2} / (p q sqrt(p+q)) becomes (c/p) (c/q) rsqrt(p+q).
constexpr double kSqrt2Pi52 = 5.9149671727956128778;
constexpr double kSqrtPiHalf = 0.88622692545275801365;  // sqrt(pi)/2

constexpr int kMaxL = 2;            // s, p, d shells
constexpr int kMaxFragAO = 232;     // AOs per fragment (packed n(n+1)/2 doubles fit in 227 KB of shared memory)
constexpr int kScfSmemMaxN = 56;    // fragment SCF: 9 n^2 doubles in shared memory up to this n
// Fragment RHF fallback: a fragment whose DIIS iteration has not converged after kScfShiftAfter
// micro-iterations continues with the virtual orbitals level-shifted by kScfLevelShift hartree.
constexpr int kScfShiftAfter = 50;
constexpr double kScfLevelShift = 0.2;
constexpr int kOrthSmemMaxN = 112;  // orthogonaliser: 2 n^2 doubles in shared memory up to this n
constexpr int kMaxLPair = 2 * kMaxL;
constexpr int kMaxLTot = 2 * kMaxLPair;

// ------------------------------------------------------------------------------------------ Boys
// FP32 grid-Taylor table for the mixed-precision J-engine: same grid, F_{m+j}(T_k)/j! for
// j = 0..4 (truncation below 0.025^5/5! ~ 8e-11, far under FP32 resolution), up to T = 30.05; above
// the table the asymptotic form is used.  The FP32 J-engine switches to the asymptotic form at
// T = 25 for L = L_P + L_Q <= 2 and at T = 30 for L = 3, 4, where the neglected exp(-T) terms are
// at most 1.4e-9 of F_L (F_2 at 25, F_4 at 30), below the FP32 resolution.
constexpr int kBoys32Order = 4;
constexpr int kBoys32Rows = 602;                  // T up to 30.05
constexpr float kFp32SwitchLow = 25.0f;           // asymptotic Boys for L <= 2 (FP32 core)
constexpr float kFp32SwitchHigh = 30.0f;          // ... for L = 3, 4
// 2/sqrt(pi) as a float pair (hi + lo): a single rounded FP32 constant would scale every quartet
// below the asymptotic switch by the same relative error (5.2e-8), a bias, not a random error.
constexpr float kTwoOverSqrtPiHi = 1.12837922573089599609375f;
constexpr float kTwoOverSqrtPiLo = -5.8635382771399236e-08f;

// Grid-Taylor table: rows T_k = k h, k = 0..kBoysRows-1; per row, for m = 0..kBoysM-1 a block of
// kBoysOrder+1 coefficients F_{m+j}(T_k)/j! (j = 0..kBoysOrder), padded to kBoysBlock doubles; the
// pad slot of block 0 holds T_k.  |T - T_k| <= h/2 = 0.025 gives a truncation error below
// 0.025^7/7! ~ 1.2e-15.  For T >= kBoysTmax the asymptotic form F_0 = sqrt(pi/T)/2,
// F_n = F_{n-1} (2n-1)/(2T) is used (neglected terms below exp(-36) ~ 2e-16).
constexpr double kBoysH = 0.05;
constexpr double kBoysInvH = 20.0;
constexpr double kBoysTmax = 36.0;
constexpr int kBoysOrder = 6;
constexpr int kBoysM = kMaxLTot + 1;              // m = 0..8
constexpr int kBoysBlock = 8;
constexpr int kBoysRowLen = kBoysM * kBoysBlock;  // 72 doubles
constexpr int kBoysRows = 732;                    // covers T up to 36.55

// float -> double by exponent re-biasing on the integer pipe (no FP64 instruction).  Zero and
// subnormal floats give 0; Inf and NaN give NaN.
__device__ __forceinline__ double f2d(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned ex = (u >> 23) & 0xffu, man = u & 0x7fffffu, sign = u & 0x80000000u;
    unsigned hi = sign | ((ex + 896u) << 20) | (man >> 3);
    unsigned lo = man << 29;
    if (ex == 0u) { hi = sign; lo = 0u; }
    if (ex == 255u) { hi = 0x7ff80000u; lo = 0u; }
    return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ double f2d(double v) { return v; }

// -------------------------------------------------------------------------------- Hermite indexing
// Hermite indices (t,u,v) with t+u+v <= L, ordered by level s = t+u+v, then t descending, then u
// descending (the Cartesian lexicographic order of each level).
__host__ __device__ constexpr int nh(int L) { return (L + 1) * (L + 2) * (L + 3) / 6; }
__host__ __device__ constexpr int ncart(int l) { return (l + 1) * (l + 2) / 2; }
__host__ __device__ constexpr int hidx(int t, int u, int v)
{
    return (t + u + v) * (t + u + v + 1) * (t + u + v + 2) / 6 + (u + v) * (u + v + 1) / 2 + v;
}
struct TUV { int t, u, v; };
__host__ __device__ constexpr TUV htuv(int idx)
{
    int s = 0;
    while (nh(s) <= idx) ++s;
    int r = idx - (s > 0 ? nh(s - 1) : 0);
    int t = s;
    while (r >= s - t + 1) { r -= s - t + 1; --t; }
    int u = s - t - r;
    return TUV{t, u, s - t - u};
}
// Cartesian component k of angular momentum l (lexicographic: xx, xy, xz, yy, yz, zz)
// Row-major upper-triangle index of the AO pair (i, j), either order: i' = min, j' = max,
// i' n - i'(i'-1)/2 + (j' - i').
__host__ __device__ inline int64_t pair_pack(int i, int j, int n)
{
    const int a = i < j ? i : j, b = i < j ? j : i;
    return (int64_t)a * n - (int64_t)a * (a - 1) / 2 + (b - a);
}

__host__ __device__ inline void cart_of(int l, int k, int& x, int& y, int& z)
{
    int n = 0;
    for (int a = l; a >= 0; --a)
        for (int b = l - a; b >= 0; --b) {
            if (n == k) { x = a; y = b; z = l - a - b; return; }
            ++n;
        }
    x = y = z = 0;
}

// ------------------------------------------------------------------------------------------ Boys (FP64)
// F_0..F_L at T (FP64), table path for T < kBoysTmax.  kidx is the nearest grid row (computed from
// an FP32 estimate of T; any row within h/2 + 1e-4 of T keeps the error bound).
template <int L>
__device__ __forceinline__ void boys_fp64(const double* __restrict__ table, double T, int kidx, double* F)
{
    if (kidx < kBoysRows - 1) {
        const double* row = table + (size_t)kidx * kBoysRowLen;
        const double Tk = __ldg(row + kBoysOrder + 1);
        const double d = Tk - T;
#pragma unroll
        for (int m = 0; m <= L; ++m) {
            const double* c = row + m * kBoysBlock;
            double2 c01 = __ldg(reinterpret_cast<const double2*>(c));
            double2 c23 = __ldg(reinterpret_cast<const double2*>(c + 2));
            double2 c45 = __ldg(reinterpret_cast<const double2*>(c + 4));
            double c6 = __ldg(c + 6);
            double f = fma(d, c6, c45.y);
            f = fma(d, f, c45.x);
            f = fma(d, f, c23.y);
            f = fma(d, f, c23.x);
            f = fma(d, f, c01.y);
            F[m] = fma(d, f, c01.x);
        }
    } else {
        const double rt = rsqrt(T);
        const double half_inv_T = 0.5 * rt * rt;
        F[0] = kSqrtPiHalf * rt;
#pragma unroll
        for (int m = 1; m <= L; ++m) F[m] = F[m - 1] * ((2.0 * m - 1.0) * half_inv_T);
    }
}

// The hardware estimate of 1/sqrt(x) (rsqrt.approx.ftz: normal inputs only, which holds for every
// argument here), without the library's subnormal-input handling.
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 1/sqrt(x) in FP32: the hardware estimate refined by one Newton step y (3 - x y^2) / 2, with the
// residual 1 - x y^2 formed by an FMA, so that the result is within about one unit in the last place
// and its error has no systematic sign (a biased 1/R would shift the whole long-range Coulomb field).
__device__ __forceinline__ float rsqrt_nr(float x)
{
    const float y = rsqrt_approx(x);
    const float h = x * y;
    const float e = fmaf(-h, y, 1.0f);
    return fmaf(0.5f * y, e, y);
}

// F_0..F_L at T in FP32 (mixed-precision core).
template <int L>
__device__ __forceinline__ void boys_fp32(const float* __restrict__ table, float T, float* F)
{
    // the row index is clamped to the table on both sides, whatever T is (T < 0 or NaN: row 0)
    const int k = (int)(fmaxf(fminf(T, (float)(kBoys32Rows - 1) * (float)kBoysH), 0.0f) * (float)kBoysInvH + 0.5f);
    if (k < kBoys32Rows - 1) {
        const float* row = table + (size_t)k * kBoysRowLen;
        const float d = __ldg(row + kBoys32Order + 3) - T;
#pragma unroll
        for (int m = 0; m <= L; ++m) {
            const float4 c = __ldg(reinterpret_cast<const float4*>(row + m * kBoysBlock));
            const float c4 = __ldg(row + m * kBoysBlock + 4);
            F[m] = fmaf(d, fmaf(d, fmaf(d, fmaf(d, c4, c.w), c.z), c.y), c.x);
        }
    } else {
        // refined reciprocal square root: the far-field quartets of every partner share its error
        const float rt = rsqrt_nr(T);
        const float half_inv_T = 0.5f * rt * rt;
        F[0] = (float)kSqrtPiHalf * rt;
#pragma unroll
        for (int m = 1; m <= L; ++m) F[m] = F[m - 1] * ((2.0f * m - 1.0f) * half_inv_T);
    }
}

// Below the asymptotic switch, the unit-normalised Hermite base of the FP32 core:
// (2/sqrt(pi)) sqrt(alpha) F_n(T) (-2 alpha)^n, n = 0..L, alpha = pq/(p+q), T = alpha R^2.  Kept out
// of line so that the common (asymptotic) path of the quartet loop carries none of its instructions.
template <int L>
struct Base32 {
    float v[L + 1];
};
template <int L>
__device__ __noinline__ Base32<L> fp32_table_base(const float* __restrict__ boys32, float pq, float sq, float R2)
{
    Base32<L> b;
    const float r = rsqrt_nr(sq);
    const float alpha = pq * (r * r);
    float F[L + 1];
    boys_fp32<L>(boys32, alpha * R2, F);
    const float sa = alpha * rsqrt_nr(alpha);
    float pre = fmaf(kTwoOverSqrtPiHi, sa, kTwoOverSqrtPiLo * sa);
    const float m2a = -2.0f * alpha;
#pragma unroll
    for (int n = 0; n <= L; ++n) {
        b.v[n] = pre * F[n];
        pre *= m2a;
    }
    return b;
}

// 1/sqrt(x) in FP64 from an FP32 estimate s of relative error e0 (up to ~1e-5): one step of the
// third-order iteration y = s (1 + e/2 + 3 e^2/8), e = 1 - x s^2 (the binomial series of (1 - e)^{-1/2}
// to second order), truncation error 5 e0^3 / 16, below the FP64 resolution.  Five FP64 operations.
__device__ __forceinline__ double rsqrt_from_seed(double x, float seed)
{
    const double s = f2d(seed);
    const double h = x * s;
    const double e = fma(-h, s, 1.0);
    const double t = fma(0.375, e, 0.5);
    return fma(s * e, t, s);
}

// Knuth's two-sum accumulation (error-free transformation of hi + a): hi becomes the rounded sum and
// lo collects the rounding errors, so that hi + lo carries the running sum to ~2^-48.
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float a)
{
    const float s = hi + a;
    const float bp = s - hi;
    const float e = (hi - (s - bp)) + (a - bp);
    hi = s;
    lo += e;
}

__device__ __forceinline__ int boys_row(float Tf)
{
    // clamped to the table on both sides: T >= Tmax + h/2 maps to the last row, which selects the
    // asymptotic branch; T < 0 or NaN (never produced by valid pair data) to row 0
    float k = fmaxf(fminf(Tf, (float)(kBoysRows - 1) * (float)kBoysH), 0.0f) * (float)kBoysInvH + 0.5f;
    return (int)k;
}

// Runtime-L variant for the non-hot kernels (one-electron, Schwarz, intra-fragment).
__device__ inline void boys_fp64_rt(const double* __restrict__ table, double T, int L, double* F)
{
    int k = (int)(fmax(fmin(T, (kBoysRows - 1) * kBoysH), 0.0) * kBoysInvH + 0.5);
    if (k < kBoysRows - 1) {
        const double* row = table + (size_t)k * kBoysRowLen;
        const double d = row[kBoysOrder + 1] - T;
        for (int m = 0; m <= L; ++m) {
            const double* c = row + m * kBoysBlock;
            double f = c[kBoysOrder];
            for (int j = kBoysOrder - 1; j >= 0; --j) f = fma(d, f, c[j]);
            F[m] = f;
        }
    } else {
        double rt = rsqrt(T);
        double hi = 0.5 * rt * rt;
        F[0] = kSqrtPiHalf * rt;
        for (int m = 1; m <= L; ++m) F[m] = F[m - 1] * ((2.0 * m - 1.0) * hi);
    }
}

// ------------------------------------------------------------------------------------------ MD R
// In-place Hermite recursion: on entry base[n] = (-2 alpha)^n F_n(T) * prefactor, n = 0..L; on exit
// R[hidx(t,u,v)] = R^{(0)}_{tuv} for t+u+v <= L, using
//   R^{(n)}_{t+1,u,v} = t R^{(n+1)}_{t-1,u,v} + X_PQ R^{(n+1)}_{t,u,v}   (and the same in u, v).
// Sweeping n from L-1 down to 0 and each level from high to low lets one array hold R^{(n+1)} of the
// lower levels while R^{(n)} of the higher levels is written.
namespace detail {
// One level sweep of md_R at order N, for Hermite index IDX down to 1 (compile-time recursion so that
// every R index is a constant and R stays in registers, or at constant offsets of a shared slice).
template <int IDX, typename Real, typename Arr>
struct MdRStep {
    static __device__ __forceinline__ void run(Arr R, Real X, Real Y, Real Z)
    {
        constexpr TUV c = htuv(IDX);
        Real v;
        if constexpr (c.t > 0) {
            v = X * R[hidx(c.t - 1, c.u, c.v)];
            if constexpr (c.t > 1) v = fma(Real(c.t - 1), R[hidx(c.t - 2, c.u, c.v)], v);
        } else if constexpr (c.u > 0) {
            v = Y * R[hidx(c.t, c.u - 1, c.v)];
            if constexpr (c.u > 1) v = fma(Real(c.u - 1), R[hidx(c.t, c.u - 2, c.v)], v);
        } else {
            v = Z * R[hidx(c.t, c.u, c.v - 1)];
            if constexpr (c.v > 1) v = fma(Real(c.v - 1), R[hidx(c.t, c.u, c.v - 2)], v);
        }
        R[IDX] = v;
        MdRStep<IDX - 1, Real, Arr>::run(R, X, Y, Z);
    }
};
template <typename Real, typename Arr>
struct MdRStep<0, Real, Arr> {
    static __device__ __forceinline__ void run(Arr, Real, Real, Real) {}
};
template <int L, int N, typename Real, typename Arr>
struct MdRLevel {
    static __device__ __forceinline__ void run(Arr R, const Real* base, Real X, Real Y, Real Z)
    {
        MdRStep<nh(L - N) - 1, Real, Arr>::run(R, X, Y, Z);
        R[0] = base[N];
        MdRLevel<L, N - 1, Real, Arr>::run(R, base, X, Y, Z);
    }
};
template <int L, typename Real, typename Arr>
struct MdRLevel<L, -1, Real, Arr> {
    static __device__ __forceinline__ void run(Arr, const Real*, Real, Real, Real) {}
};
}  // namespace detail

template <int L, typename Real, typename Arr>
__device__ __forceinline__ void md_R(Arr R, const Real* base, Real X, Real Y, Real Z)
{
    R[0] = base[L];
    detail::MdRLevel<L, L - 1, Real, Arr>::run(R, base, X, Y, Z);
}

// Per-lane slice of a warp's shared buffer, element i of lane l at p[i * 32 + l] (conflict-free).
template <typename Real>
struct LaneSlice {
    Real* p;
    __device__ __forceinline__ Real& operator[](int i) const { return p[i * 32]; }
};

// Runtime-L R recursion for the non-hot kernels; R has room for nh(L) values, scratch for the
// same.  Same recurrence as md_R.
__device__ inline void md_R_rt(int L, double* R, const double* base, double X, double Y, double Z)
{
    R[0] = base[L];
    for (int n = L - 1; n >= 0; --n) {
        for (int idx = nh(L - n) - 1; idx >= 1; --idx) {
            TUV c = htuv(idx);
            double v;
            if (c.t > 0) {
                v = X * R[hidx(c.t - 1, c.u, c.v)];
                if (c.t > 1) v += (c.t - 1) * R[hidx(c.t - 2, c.u, c.v)];
            } else if (c.u > 0) {
                v = Y * R[hidx(c.t, c.u - 1, c.v)];
                if (c.u > 1) v += (c.u - 1) * R[hidx(c.t, c.u - 2, c.v)];
            } else {
                v = Z * R[hidx(c.t, c.u, c.v - 1)];
                if (c.v > 1) v += (c.v - 1) * R[hidx(c.t, c.u, c.v - 2)];
            }
            R[idx] = v;
        }
        R[0] = base[n];
    }
}

// ------------------------------------------------------------------------------------------ MD E
// 1D Hermite expansion coefficients E^{ij}_t (i <= la, j <= lb, t <= i+j) of
// x_A^i x_B^j exp(-a x_A^2 - b x_B^2) = K_x sum_t E^{ij}_t Lambda_t(x_P), with K_x factored out
// (E^{00}_0 = 1):
//   E^{i+1,j}_t = E^{ij}_{t-1}/(2p) + X_PA E^{ij}_t + (t+1) E^{ij}_{t+1}
//   E^{i,j+1}_t = E^{ij}_{t-1}/(2p) + X_PB E^{ij}_t + (t+1) E^{ij}_{t+1}
// E is indexed [i][j][t] with fixed strides (3, 3, 5).
__device__ __forceinline__ void md_E1(int la, int lb, double p, double XPA, double XPB, double (*E)[3][5])
{
    const double h = 0.5 / p;
    for (int i = 0; i <= la; ++i)
        for (int j = 0; j <= lb; ++j)
            for (int t = 0; t < 5; ++t) E[i][j][t] = 0.0;
    E[0][0][0] = 1.0;
    for (int i = 0; i < la; ++i)
        for (int t = 0; t <= i + 1; ++t) {
            double v = XPA * (t <= i ? E[i][0][t] : 0.0);
            if (t > 0) v += h * E[i][0][t - 1];
            if (t + 1 <= i) v += (t + 1) * E[i][0][t + 1];
            E[i + 1][0][t] = v;
        }
    for (int i = 0; i <= la; ++i)
        for (int j = 0; j < lb; ++j)
            for (int t = 0; t <= i + j + 1; ++t) {
                double v = XPB * (t <= i + j ? E[i][j][t] : 0.0);
                if (t > 0) v += h * E[i][j][t - 1];
                if (t + 1 <= i + j) v += (t + 1) * E[i][j][t + 1];
                E[i][j + 1][t] = v;
            }
}

// Shell-level primitive normalisation (2a/pi)^{3/4} (4a)^{l/2}.
__device__ inline double prim_norm(double a, int l)
{
    double n = pow(2.0 * a / kPi, 0.75);
    for (int k = 0; k < l; ++k) n *= sqrt(4.0 * a);
    return n;
}

// ------------------------------------------------------------------------------------------ errors
// Device error flags (bit mask), read by the host after a launch sequence.
enum : int {
    kErrNumeric = 1,   // NaN/Inf in a matrix or energy
    kErrBounds = 4,    // an index failed a bounds check
    kErrNotConv = 8,   // a fragment RHF hit its iteration limit
};

}  // namespace fef
