// fef_fragment_rhf_noalloc: the batched fragment RHF (canonical orthogonaliser + the device SCF loop
// of scf.cu) for callers that cannot allocate device memory.
//
// Who cannot allocate: host codes that own every byte of device memory themselves (a molecular
// dynamics or embedding driver with a fixed memory budget or its own pool), and callers that must not
// pay for, or serialise on, cudaMalloc/cudaFree in a time step.  This entry point therefore takes all
// inputs and outputs from the caller and keeps its own working memory (orthogonalisers, DIIS history,
// per-fragment offsets, status flag) in one file-scope device array of fixed size, g_noalloc_scratch
// (16 MiB).  Every GPU that loads the library holds that array until the process exits.
//
// Set-up: the first call on each device, with that device current, resolves the array's device
// address with cudaGetSymbolAddress and caches it; make that first call before any stream capture
// begins.  All calls share the array and it keeps the previous call's contents, so calls whose device
// work overlaps (two streams, two host threads) race on it.  The status flag is cleared at the start
// of every call; the call then reads it back and synchronises the stream before it returns.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"
#include "internal.hpp"

namespace fef {

void set_global_error(const char* msg);  // api.cu: message for fef_last_error(NULL)

constexpr size_t kNoAllocBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char* g_noalloc_ptr[kMaxDevices] = {};

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Packed-block offsets of the caller's matrices: moff[x] = sum_{y<x} n_y^2, eoff[x] = sum n_y^4.
__global__ void k_noalloc_offsets(int n_frag, const int* nao, int64_t* moff, int64_t* eoff)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int64_t m = 0, e = 0;
    for (int x = 0; x < n_frag; ++x) {
        moff[x] = m;
        eoff[x] = e;
        int64_t n = nao[x];
        m += n * n;
        e += n * n * n * n;
    }
    moff[n_frag] = m;
    eoff[n_frag] = e;
}

fef_status fail(fef_status st, const char* msg)
{
    set_global_error(msg);
    return st;
}

}  // namespace

}  // namespace fef

using namespace fef;

extern "C" fef_status fef_fragment_rhf_noalloc(int32_t n_frag, const int32_t* n_ao, const int32_t* n_occ,
                                               const double* e_nn, const double* S, const double* h,
                                               const double* omega, const double* eri_c, const double* D_start,
                                               double* D_out, double* F_out, double* E_scf,
                                               const fef_options* opt, void* cuda_stream)
{
    if (n_frag < 1 || n_frag > 65535) return fail(FEF_ERR_ARG, "fef_fragment_rhf_noalloc: n_frag must be 1..65535");
    if (!n_ao || !n_occ || !e_nn || !S || !h || !eri_c || !D_out || !F_out || !E_scf)
        return fail(FEF_ERR_ARG, "fef_fragment_rhf_noalloc: NULL input or output pointer");
    fef_options o;
    if (opt) o = *opt; else fef_default_options(&o);
    if (o.diis_size < 1 || o.diis_size > 8 || o.max_micro < 1)
        return fail(FEF_ERR_ARG, "fef_fragment_rhf_noalloc: diis_size must be 1..8 and max_micro >= 1");
    int max_n = 0;
    int64_t sum_n2 = 0;
    for (int x = 0; x < n_frag; ++x) {
        if (n_ao[x] < 1 || n_ao[x] > 56)
            return fail(FEF_ERR_ARG, "fef_fragment_rhf_noalloc: every n_ao must be 1..56");
        if (n_occ[x] < 0 || n_occ[x] > n_ao[x])
            return fail(FEF_ERR_ARG, "fef_fragment_rhf_noalloc: n_occ must be 0..n_ao");
        max_n = n_ao[x] > max_n ? n_ao[x] : max_n;
        sum_n2 += (int64_t)n_ao[x] * n_ao[x];
    }
    // scratch layout: flag | nao | nocc | nmo | iters | moff | eoff | e_nn | E_int | X | DIIS
    const size_t nf = (size_t)n_frag;
    const int64_t diis_stride = 2 * (int64_t)o.diis_size * max_n * max_n;
    size_t off[11];
    size_t b = 0;
    off[0] = b; b += align256(sizeof(int));
    off[1] = b; b += align256(nf * sizeof(int));
    off[2] = b; b += align256(nf * sizeof(int));
    off[3] = b; b += align256(nf * sizeof(int));
    off[4] = b; b += align256(nf * sizeof(int));
    off[5] = b; b += align256((nf + 1) * sizeof(int64_t));
    off[6] = b; b += align256((nf + 1) * sizeof(int64_t));
    off[7] = b; b += align256(nf * sizeof(double));
    off[8] = b; b += align256(nf * sizeof(double));
    off[9] = b; b += align256((size_t)sum_n2 * sizeof(double));
    off[10] = b; b += align256(nf * (size_t)diis_stride * sizeof(double));
    if (b > kNoAllocBytes)
        return fail(FEF_ERR_ARG, "fef_fragment_rhf_noalloc: the batch needs more than the 16 MiB static scratch "
                                 "(orthogonalisers + 2*diis_size*max_n^2 doubles of DIIS history per fragment); "
                                 "split it into smaller batches");

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(FEF_ERR_CUDA, "fef_fragment_rhf_noalloc: no usable current CUDA device");
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p)
                return fail(FEF_ERR_CUDA, "fef_fragment_rhf_noalloc: cudaGetSymbolAddress of the static scratch failed");
            g_noalloc_ptr[dev] = static_cast<unsigned char*>(p);
        }
        base = g_noalloc_ptr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int* flag = reinterpret_cast<int*>(base + off[0]);
    int* nao_d = reinterpret_cast<int*>(base + off[1]);
    int* nocc_d = reinterpret_cast<int*>(base + off[2]);
    int* nmo_d = reinterpret_cast<int*>(base + off[3]);
    int* iters_d = reinterpret_cast<int*>(base + off[4]);
    int64_t* moff_d = reinterpret_cast<int64_t*>(base + off[5]);
    int64_t* eoff_d = reinterpret_cast<int64_t*>(base + off[6]);
    double* enn_d = reinterpret_cast<double*>(base + off[7]);
    double* eint_d = reinterpret_cast<double*>(base + off[8]);
    double* X_d = reinterpret_cast<double*>(base + off[9]);
    double* diis_d = reinterpret_cast<double*>(base + off[10]);

    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(nao_d, n_ao, nf * sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(nocc_d, n_occ, nf * sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(enn_d, e_nn, nf * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        k_noalloc_offsets<<<1, 32, 0, s>>>(n_frag, nao_d, moff_d, eoff_d);
        note_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && D_start && D_start != D_out)
        e = cudaMemcpyAsync(D_out, D_start, (size_t)sum_n2 * sizeof(double), cudaMemcpyDeviceToDevice, s);
    Dev d{};
    d.n_frag = n_frag;
    d.max_nao = max_n;
    d.frag_nao = nao_d;
    d.frag_nocc = nocc_d;
    d.frag_moff = moff_d;
    d.frag_eoff = eoff_d;
    d.err_flag = flag;
    if (e == cudaSuccess) e = launch_orthogonaliser(d, S, X_d, nmo_d, 1e-7, max_n, s);
    ScfArgs a{};
    a.h = h;
    a.omega = omega;
    a.S = S;
    a.X = X_d;
    a.nmo = nmo_d;
    a.eric = eri_c;
    a.e_nn = enn_d;
    a.D = D_out;
    a.F = F_out;
    a.diis_F = diis_d;
    a.diis_stride = diis_stride;
    a.E_scf = E_scf;
    a.E_int = eint_d;
    a.iters = iters_d;
    a.have_start = D_start ? 1 : 0;
    a.max_iter = o.max_micro;
    a.diis_size = o.diis_size;
    a.e_tol = o.micro_e_tol;
    a.comm_tol = o.micro_comm_tol;
    if (e == cudaSuccess) e = launch_fragment_scf(d, a, max_n, s);
    int hflag = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(FEF_ERR_CUDA, cudaGetErrorString(e));
    if (hflag & kErrNumeric) return fail(FEF_ERR_NUMERIC, "fef_fragment_rhf_noalloc: NaN/Inf in a fragment SCF");
    if (hflag & kErrBounds)
        return fail(FEF_ERR_ARG, "fef_fragment_rhf_noalloc: a device bounds check failed (inputs inconsistent "
                                 "with n_ao)");
    if (hflag & kErrNotConv)
        return fail(FEF_ERR_NOT_CONVERGED, "fef_fragment_rhf_noalloc: a fragment RHF hit max_micro");
    if (hflag != 0) return fail(FEF_ERR_CUDA, "fef_fragment_rhf_noalloc: unexpected device status flag");
    return FEF_OK;
}
