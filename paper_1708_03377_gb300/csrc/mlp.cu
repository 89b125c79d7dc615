// Warm-start network: a 3-layer perceptron H1 = tanh(X W1 + b1), H2 = tanh(H1 W2 + b2),
// Y = H2 W3 + b3, trained with mean squared error and Adam (Kingma & Ba 2015), FP32 weights with
// FP32 accumulation.  The paper has no learned component; this network predicts the change of a
// fragment's density from its isolated-fragment RHF density in the field of its environment, to
// start the FEF iterations closer to self-consistency.
//
// Parameters are one flat buffer: W1 (n_in x n_h, row-major), b1, W2 (n_h x n_h), b2,
// W3 (n_h x n_out), b3.  Matrices of activations are row-major [batch x width].
#include <algorithm>
#include <cmath>
#include <random>
#include <string>
#include <vector>

#include "internal.hpp"

struct fef_mlp {
    int n_in = 0, n_h = 0, n_out = 0;
    int64_t n_par = 0;
    cudaStream_t stream = nullptr;
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    int cap = 0;
    float *Xb = nullptr, *Tb = nullptr, *H1 = nullptr, *H2 = nullptr, *Y = nullptr, *dY = nullptr, *dZ2 = nullptr,
          *dZ1 = nullptr;
    int* perm = nullptr;
    int perm_cap = 0;
    double* loss_acc = nullptr;
    float *in_shift = nullptr, *in_scale = nullptr, *out_shift = nullptr, *out_scale = nullptr;
    bool scaled = false;
    int64_t step = 0;
    unsigned long long seed = 0;
    std::string last_error;
};

namespace fef {
namespace {

void set_err(fef_mlp* m, const std::string& s) { if (m) m->last_error = s; }

constexpr int TILE = 16;

// C[M x N] = op(A) op(B) (+ bias[n]) then epilogue: 0 none, 1 tanh, 2 multiply by (1 - H^2).
// TA = 1: A is stored K x M (use A^T); TB = 1: B is stored N x K (use B^T).
template <int TA, int TB, int EPI>
__global__ void k_gemm(int M, int N, int K, const float* __restrict__ A, const float* __restrict__ B,
                       const float* __restrict__ bias, const float* __restrict__ H, float* __restrict__ C)
{
    __shared__ float As[TILE][TILE + 1], Bs[TILE][TILE + 1];
    const int ty = threadIdx.y, tx = threadIdx.x;
    const int row = blockIdx.y * TILE + ty, col = blockIdx.x * TILE + tx;
    float acc = 0.0f;
    for (int k0 = 0; k0 < K; k0 += TILE) {
        const int ar = blockIdx.y * TILE + ty, ac = k0 + tx;
        As[ty][tx] = (ar < M && ac < K) ? (TA ? A[(size_t)ac * M + ar] : A[(size_t)ar * K + ac]) : 0.0f;
        const int br = k0 + ty, bc = blockIdx.x * TILE + tx;
        Bs[ty][tx] = (br < K && bc < N) ? (TB ? B[(size_t)bc * K + br] : B[(size_t)br * N + bc]) : 0.0f;
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TILE; ++kk) acc = fmaf(As[ty][kk], Bs[kk][tx], acc);
        __syncthreads();
    }
    if (row < M && col < N) {
        if (bias) acc += bias[col];
        if (EPI == 1) acc = tanhf(acc);
        if (EPI == 2) {
            const float h = H[(size_t)row * N + col];
            acc *= 1.0f - h * h;
        }
        C[(size_t)row * N + col] = acc;
    }
}

template <int TA, int TB, int EPI>
void gemm(cudaStream_t s, int M, int N, int K, const float* A, const float* B, const float* bias, const float* H,
          float* C)
{
    dim3 b(TILE, TILE), g((N + TILE - 1) / TILE, (M + TILE - 1) / TILE);
    k_gemm<TA, TB, EPI><<<g, b, 0, s>>>(M, N, K, A, B, bias, H, C);
    note_launches(1);
}

// out[n] = sum over rows of Z[rows x N]
__global__ void k_colsum(int rows, int N, const float* __restrict__ Z, float* out)
{
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.0f;
    for (int r = 0; r < rows; ++r) s += Z[(size_t)r * N + n];
    out[n] = s;
}

// dY = 2 (Y - T) / (N n_out); loss_acc += sum (Y - T)^2
__global__ void k_mse(int64_t n, const float* __restrict__ Y, const float* __restrict__ T, float scale, float* dY,
                      double* loss_acc)
{
    double part = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float r = Y[i] - T[i];
        if (dY) dY[i] = 2.0f * r * scale;
        part += (double)r * r;
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss_acc, part);
}

__global__ void k_adam(int64_t n, float* theta, const float* g, float* m, float* v, float lr, float b1, float b2,
                       float c1, float c2)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
    }
}

// splitmix64 (Steele, Lea & Flood 2014): counter-based generator for the initial weights.
__device__ inline unsigned long long splitmix64(unsigned long long z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Glorot-uniform weights, zero biases.
__global__ void k_init(float* theta, int n_in, int n_h, int n_out, unsigned long long seed)
{
    const int64_t sizes[6] = {(int64_t)n_in * n_h, n_h, (int64_t)n_h * n_h, n_h, (int64_t)n_h * n_out, n_out};
    const int fan_in[3] = {n_in, n_h, n_h}, fan_out[3] = {n_h, n_h, n_out};
    int64_t total = 0;
    for (int k = 0; k < 6; ++k) total += sizes[k];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t o = i;
        int part = 0;
        while (o >= sizes[part]) o -= sizes[part++];
        if (part & 1) {
            theta[i] = 0.0f;
        } else {
            const int l = part / 2;
            const float a = sqrtf(6.0f / (float)(fan_in[l] + fan_out[l]));
            const unsigned long long r = splitmix64(seed ^ (unsigned long long)i * 0xD1B54A32D192ED03ull);
            const float u = (float)((r >> 40) * (1.0 / 16777216.0));  // 24 random bits in [0, 1)
            theta[i] = (2.0f * u - 1.0f) * a;
        }
    }
}

__global__ void k_gather(int rows, int width, const int* __restrict__ perm, int off, const float* __restrict__ src,
                         float* dst)
{
    int64_t n = (int64_t)rows * width;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / width), c = (int)(i % width);
        dst[i] = src[(size_t)perm[off + r] * width + c];
    }
}

// X <- (X - shift) / scale per column (in place) or Y <- shift + scale Y
__global__ void k_affine(int64_t n, int width, float* X, const float* shift, const float* scale, int inverse)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % width);
        X[i] = inverse ? shift[c] + scale[c] * X[i] : (X[i] - shift[c]) / scale[c];
    }
}

cudaError_t ensure_cap(fef_mlp* m, int rows)
{
    if (rows <= m->cap) return cudaSuccess;
    float** bufs[] = {&m->Xb, &m->Tb, &m->H1, &m->H2, &m->Y, &m->dY, &m->dZ2, &m->dZ1};
    for (float** b : bufs)
        if (*b) cudaFree(*b);
    const int w[] = {m->n_in, m->n_out, m->n_h, m->n_h, m->n_out, m->n_out, m->n_h, m->n_h};
    for (int k = 0; k < 8; ++k) {
        cudaError_t e = cudaMalloc(bufs[k], sizeof(float) * (size_t)rows * w[k]);
        if (e != cudaSuccess) return e;
    }
    m->cap = rows;
    return cudaSuccess;
}

// forward of rows x n_in (already standardised) into m->H1, m->H2, m->Y
void forward(fef_mlp* m, int rows, const float* X, cudaStream_t st)
{
    const float* W1 = m->theta;
    const float* b1 = W1 + (size_t)m->n_in * m->n_h;
    const float* W2 = b1 + m->n_h;
    const float* b2 = W2 + (size_t)m->n_h * m->n_h;
    const float* W3 = b2 + m->n_h;
    const float* b3 = W3 + (size_t)m->n_h * m->n_out;
    gemm<0, 0, 1>(st, rows, m->n_h, m->n_in, X, W1, b1, nullptr, m->H1);
    gemm<0, 0, 1>(st, rows, m->n_h, m->n_h, m->H1, W2, b2, nullptr, m->H2);
    gemm<0, 0, 0>(st, rows, m->n_out, m->n_h, m->H2, W3, b3, nullptr, m->Y);
}

// loss and gradient of rows x (X, T) into m->grad; adds sum of squares to *m->loss_acc
void backward(fef_mlp* m, int rows, const float* X, const float* T, float scale)
{
    const int ni = m->n_in, nh = m->n_h, no = m->n_out;
    const float* W1 = m->theta;
    const float* W2 = W1 + (size_t)ni * nh + nh;
    const float* W3 = W2 + (size_t)nh * nh + nh;
    float* gW1 = m->grad;
    float* gb1 = gW1 + (size_t)ni * nh;
    float* gW2 = gb1 + nh;
    float* gb2 = gW2 + (size_t)nh * nh;
    float* gW3 = gb2 + nh;
    float* gb3 = gW3 + (size_t)nh * no;
    const int64_t ny = (int64_t)rows * no;
    k_mse<<<(unsigned)std::min<int64_t>((ny + 255) / 256, 1024), 256, 0, m->stream>>>(ny, m->Y, T, scale, m->dY,
                                                                                      m->loss_acc);
    note_launches(1);
    gemm<1, 0, 0>(m->stream, nh, no, rows, m->H2, m->dY, nullptr, nullptr, gW3);     // dW3 = H2^T dY
    k_colsum<<<(no + 127) / 128, 128, 0, m->stream>>>(rows, no, m->dY, gb3);
    note_launches(1);
    gemm<0, 1, 2>(m->stream, rows, nh, no, m->dY, W3, nullptr, m->H2, m->dZ2);       // dZ2 = dY W3^T (1-H2^2)
    gemm<1, 0, 0>(m->stream, nh, nh, rows, m->H1, m->dZ2, nullptr, nullptr, gW2);    // dW2 = H1^T dZ2
    k_colsum<<<(nh + 127) / 128, 128, 0, m->stream>>>(rows, nh, m->dZ2, gb2);
    note_launches(1);
    gemm<0, 1, 2>(m->stream, rows, nh, nh, m->dZ2, W2, nullptr, m->H1, m->dZ1);      // dZ1 = dZ2 W2^T (1-H1^2)
    gemm<1, 0, 0>(m->stream, ni, nh, rows, X, m->dZ1, nullptr, nullptr, gW1);        // dW1 = X^T dZ1
    k_colsum<<<(nh + 127) / 128, 128, 0, m->stream>>>(rows, nh, m->dZ1, gb1);
    note_launches(1);
}

}  // namespace
}  // namespace fef

using namespace fef;

extern "C" fef_status fef_mlp_create(int32_t n_in, int32_t n_hidden, int32_t n_out, uint64_t seed, void* stream,
                                     fef_mlp** out)
{
    if (!out || n_in < 1 || n_hidden < 1 || n_out < 1 || n_in > 4096 || n_hidden > 4096 || n_out > 4096)
        return FEF_ERR_ARG;
    fef_mlp* m = new fef_mlp();
    m->n_in = n_in;
    m->n_h = n_hidden;
    m->n_out = n_out;
    m->n_par = (int64_t)n_in * n_hidden + n_hidden + (int64_t)n_hidden * n_hidden + n_hidden +
               (int64_t)n_hidden * n_out + n_out;
    m->stream = static_cast<cudaStream_t>(stream);
    m->seed = seed;
    cudaError_t e = cudaSuccess;
    float** p[] = {&m->theta, &m->grad, &m->m, &m->v};
    for (float** q : p)
        if (e == cudaSuccess) e = cudaMalloc(q, sizeof(float) * m->n_par);
    if (e == cudaSuccess) e = cudaMalloc(&m->loss_acc, sizeof(double));
    float** sc[] = {&m->in_shift, &m->in_scale, &m->out_shift, &m->out_scale};
    const int w[] = {n_in, n_in, n_out, n_out};
    for (int k = 0; k < 4; ++k)
        if (e == cudaSuccess) e = cudaMalloc(sc[k], sizeof(float) * w[k]);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->m, 0, sizeof(float) * m->n_par, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->v, 0, sizeof(float) * m->n_par, m->stream);
    if (e == cudaSuccess) {
        k_init<<<256, 256, 0, m->stream>>>(m->theta, n_in, n_hidden, n_out, seed);
        note_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) {
        fef_mlp_destroy(m);
        return FEF_ERR_CUDA;
    }
    *out = m;
    return FEF_OK;
}

extern "C" void fef_mlp_destroy(fef_mlp* m)
{
    if (!m) return;
    float* bufs[] = {m->theta, m->grad, m->m, m->v, m->Xb, m->Tb, m->H1, m->H2, m->Y, m->dY, m->dZ2, m->dZ1,
                     m->in_shift, m->in_scale, m->out_shift, m->out_scale};
    for (float* b : bufs)
        if (b) cudaFree(b);
    if (m->perm) cudaFree(m->perm);
    if (m->loss_acc) cudaFree(m->loss_acc);
    delete m;
}

extern "C" fef_status fef_mlp_params(fef_mlp* m, float* params, int64_t* n_params, int32_t set)
{
    if (!m) return FEF_ERR_ARG;
    if (n_params) *n_params = m->n_par;
    if (!params) return FEF_OK;
    cudaError_t e = set ? cudaMemcpyAsync(m->theta, params, sizeof(float) * m->n_par, cudaMemcpyHostToDevice, m->stream)
                        : cudaMemcpyAsync(params, m->theta, sizeof(float) * m->n_par, cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) { set_err(m, cudaGetErrorString(e)); return FEF_ERR_CUDA; }
    if (set) {
        m->step = 0;
        cudaMemsetAsync(m->m, 0, sizeof(float) * m->n_par, m->stream);
        cudaMemsetAsync(m->v, 0, sizeof(float) * m->n_par, m->stream);
    }
    return FEF_OK;
}

extern "C" fef_status fef_mlp_set_scaling(fef_mlp* m, const float* in_shift, const float* in_scale,
                                          const float* out_shift, const float* out_scale)
{
    if (!m || !in_shift || !in_scale || !out_shift || !out_scale) return FEF_ERR_ARG;
    cudaError_t e = cudaMemcpyAsync(m->in_shift, in_shift, sizeof(float) * m->n_in, cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->in_scale, in_scale, sizeof(float) * m->n_in, cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->out_shift, out_shift, sizeof(float) * m->n_out, cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->out_scale, out_scale, sizeof(float) * m->n_out, cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) { set_err(m, cudaGetErrorString(e)); return FEF_ERR_CUDA; }
    m->scaled = true;
    return FEF_OK;
}

extern "C" fef_status fef_mlp_loss_grad(fef_mlp* m, const float* X, const float* T, int32_t n, float* loss,
                                        float* grad)
{
    if (!m || !X || !T || n < 1) return FEF_ERR_ARG;
    cudaError_t e = ensure_cap(m, n);
    if (e != cudaSuccess) { set_err(m, cudaGetErrorString(e)); return FEF_ERR_CUDA; }
    cudaMemsetAsync(m->loss_acc, 0, sizeof(double), m->stream);
    forward(m, n, X, m->stream);
    backward(m, n, X, T, 1.0f / ((float)n * m->n_out));
    double acc = 0.0;
    e = cudaMemcpyAsync(&acc, m->loss_acc, sizeof(double), cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess && grad)
        e = cudaMemcpyAsync(grad, m->grad, sizeof(float) * m->n_par, cudaMemcpyDeviceToDevice, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) { set_err(m, cudaGetErrorString(e)); return FEF_ERR_CUDA; }
    if (loss) *loss = (float)(acc / ((double)n * m->n_out));
    return FEF_OK;
}

extern "C" fef_status fef_mlp_train(fef_mlp* m, const float* X, const float* T, int32_t n, int32_t epochs,
                                    int32_t batch, float lr, float* final_loss)
{
    if (!m || !X || !T || n < 1 || epochs < 1 || batch < 1 || !(lr > 0.0f)) return FEF_ERR_ARG;
    batch = std::min(batch, n);
    cudaError_t e = ensure_cap(m, batch);
    if (e == cudaSuccess && m->perm_cap < n) {
        if (m->perm) cudaFree(m->perm);
        e = cudaMalloc(&m->perm, sizeof(int) * n);
        m->perm_cap = n;
    }
    if (e != cudaSuccess) { set_err(m, cudaGetErrorString(e)); return FEF_ERR_CUDA; }
    std::vector<int> perm(n);
    std::mt19937_64 rng(m->seed + 0x5851F42D4C957F2Dull);
    double epoch_loss = 0.0;
    for (int ep = 0; ep < epochs; ++ep) {
        for (int i = 0; i < n; ++i) perm[i] = i;
        std::shuffle(perm.begin(), perm.end(), rng);
        e = cudaMemcpyAsync(m->perm, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, m->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(m->loss_acc, 0, sizeof(double), m->stream);
        if (e != cudaSuccess) break;
        for (int off = 0; off < n; off += batch) {
            const int rows = std::min(batch, n - off);
            k_gather<<<128, 256, 0, m->stream>>>(rows, m->n_in, m->perm, off, X, m->Xb);
            k_gather<<<128, 256, 0, m->stream>>>(rows, m->n_out, m->perm, off, T, m->Tb);
            note_launches(2);
            forward(m, rows, m->Xb, m->stream);
            backward(m, rows, m->Xb, m->Tb, 1.0f / ((float)rows * m->n_out));
            ++m->step;
            const float b1 = 0.9f, b2 = 0.999f;
            k_adam<<<256, 256, 0, m->stream>>>(m->n_par, m->theta, m->grad, m->m, m->v, lr, b1, b2,
                                               1.0f - powf(b1, (float)m->step), 1.0f - powf(b2, (float)m->step));
            note_launches(1);
        }
        double acc = 0.0;
        e = cudaMemcpyAsync(&acc, m->loss_acc, sizeof(double), cudaMemcpyDeviceToHost, m->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
        if (e != cudaSuccess) break;
        epoch_loss = acc / ((double)n * m->n_out);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) { set_err(m, cudaGetErrorString(e)); return FEF_ERR_CUDA; }
    if (final_loss) *final_loss = (float)epoch_loss;
    return FEF_OK;
}

namespace fef {
// Y[n x n_out] = network(X[n x n_in]) on stream st, applying the input/output scaling when set.
// The network's scratch rows are shared: one prediction or training call at a time per network.
cudaError_t mlp_predict_device(fef_mlp* m, const float* X, float* Y, int n, cudaStream_t st)
{
    cudaError_t e = ensure_cap(m, n);
    if (e != cudaSuccess) return e;
    const float* Xin = X;
    if (m->scaled) {
        e = cudaMemcpyAsync(m->Xb, X, sizeof(float) * (size_t)n * m->n_in, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
        k_affine<<<128, 256, 0, st>>>((int64_t)n * m->n_in, m->n_in, m->Xb, m->in_shift, m->in_scale, 0);
        note_launches(1);
        Xin = m->Xb;
    }
    forward(m, n, Xin, st);
    if (m->scaled) {
        k_affine<<<128, 256, 0, st>>>((int64_t)n * m->n_out, m->n_out, m->Y, m->out_shift, m->out_scale, 1);
        note_launches(1);
    }
    e = cudaMemcpyAsync(Y, m->Y, sizeof(float) * (size_t)n * m->n_out, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
}
int mlp_n_in(const fef_mlp* m) { return m->n_in; }
int mlp_n_out(const fef_mlp* m) { return m->n_out; }
}  // namespace fef

extern "C" fef_status fef_mlp_predict(fef_mlp* m, const float* X, float* Y, int32_t n)
{
    if (!m || !X || !Y || n < 1) return FEF_ERR_ARG;
    cudaError_t e = mlp_predict_device(m, X, Y, n, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) { set_err(m, cudaGetErrorString(e)); return FEF_ERR_CUDA; }
    return FEF_OK;
}

extern "C" const char* fef_mlp_last_error(const fef_mlp* m) { return m ? m->last_error.c_str() : ""; }
