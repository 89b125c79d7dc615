// C ABI of libfef.so (include/fef.h): input validation, integer bookkeeping of shells, shell pairs,
// primitive pairs and J-engine tiles, device memory, and the orchestration of the FEF Fock build and
// FEF self-consistency (paper, "Fragment Mean Field").  All arithmetic of the method runs in the
// kernels of setup.cu, jengine.cu and scf.cu.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.hpp"

namespace fef {

struct Error {
    fef_status status;
    std::string msg;
};

static void ck(cudaError_t e, const char* what)
{
    if (e != cudaSuccess) throw Error{FEF_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e)};
}

// Device memory of a context comes from one stream-ordered memory pool per device, shared by all
// contexts and kept (up to kPoolKeepBytes) across them, so that creating and destroying contexts of
// the same size repeatedly costs no cudaMalloc/cudaFree (and no device synchronisation) after the first.
constexpr uint64_t kPoolKeepBytes = 4ull << 30;

static cudaMemPool_t device_pool(int device)
{
    static std::mutex mu;
    static std::vector<cudaMemPool_t> pools;
    std::lock_guard<std::mutex> lock(mu);
    if ((int)pools.size() <= device) pools.resize(device + 1, nullptr);
    if (!pools[device]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        cudaMemPool_t p = nullptr;
        ck(cudaMemPoolCreate(&p, &props), "memory pool");
        uint64_t keep = kPoolKeepBytes;
        ck(cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep), "memory pool");
        pools[device] = p;
    }
    return pools[device];
}

struct Buffers {
    std::vector<void*> allocs;
    cudaMemPool_t pool = nullptr;  // allocations in stream order on `as` (the context stream at creation)
    cudaStream_t as = nullptr;
    template <typename T>
    T* alloc(size_t n, const char* what)
    {
        void* p = nullptr;
        const size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
        if (pool)
            ck(cudaMallocFromPoolAsync(&p, bytes, pool, as), what);
        else
            ck(cudaMalloc(&p, bytes), what);
        allocs.push_back(p);
        return static_cast<T*>(p);
    }
    template <typename T>
    T* upload(const std::vector<T>& v, cudaStream_t s, const char* what)
    {
        T* p = alloc<T>(v.size(), what);
        if (!v.empty()) ck(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s), what);
        return p;
    }
    void release(void* p)
    {
        auto it = std::find(allocs.begin(), allocs.end(), p);
        if (it != allocs.end()) {
            if (pool)
                cudaFreeAsync(p, as);  // after the context's work on `as` that used it
            else
                cudaFree(p);
            allocs.erase(it);
        }
    }
    ~Buffers()
    {
        for (auto& g : macro_graph)
            if (g) cudaGraphExecDestroy(g);
        if (capture_stream) cudaStreamDestroy(capture_stream);
        if (jplan) jplan_destroy(jplan);
        if (stage) cudaFreeHost(stage);
        if (scf_tol_host) cudaFreeHost(scf_tol_host);
        if (pool) {
            // the context's work may run on streams the caller owns: wait for the device, then
            // return the memory to the pool
            cudaDeviceSynchronize();
            for (void* p : allocs) cudaFreeAsync(p, nullptr);
        } else {
            for (void* p : allocs) cudaFree(p);
        }
    }
    // one CUDA graph per kind of macro-iteration (fragment SCF + Fock build + read-back), built on
    // first use; launches of this library inside each graph
    cudaGraphExec_t macro_graph[3] = {};
    cudaStream_t capture_stream = nullptr;  // private stream for captures (the context stream may be the legacy one)
    bool capturing = false;
    int64_t* trf_off = nullptr;             // [2 n_pairs + 1] offsets of the nuclear trace fields
    double* trf = nullptr;                  // Hermite fields of each pair's nuclei (geometry time)
    unsigned long long* stamps = nullptr;   // [4] device timestamps of the phase marks in graph mode
    long long macro_graph_launches[3] = {};
    // pinned read-back of one macro-iteration: E_tot, error flag, E_frag[n], iters[n]
    unsigned char* stage = nullptr;
    double* scf_tol = nullptr;       // device [2]: micro-iteration thresholds of the next fragment SCF
    double* scf_tol_host = nullptr;  // pinned staging of scf_tol
    // geometry-time data
    double *S = nullptr, *h = nullptr, *X = nullptr, *Venv = nullptr, *eric = nullptr, *boys = nullptr;
    double* scf_ws = nullptr;  // fragment-SCF workspace for fragments above kScfSmemMaxN AOs
    int* scf_small = nullptr;  // fragments of the one-block-per-fragment SCF launch (when some are large)
    int* scf_big = nullptr;    // fragments above kScfSmemMaxN AOs: one thread-block cluster each
    int n_scf_small = 0, n_scf_big = 0;
    double* gap = nullptr;     // [n_frag] HOMO-LUMO gap of each fragment's last Roothaan step
    // far field (opt.far_field): moment integrals, nuclear moments and centroids (geometry time);
    // multipoles, far potentials and half pair energies per fragment (per build)
    double *far_M = nullptr, *far_Mnuc = nullptr, *far_cen = nullptr;
    double *far_mult = nullptr, *far_pot = nullptr, *far_E = nullptr;
    bool far_on = false;       // far-field terms in every build (opt.far_field with a cutoff)
    double* omega_mp = nullptr;  // learned start: multipole estimate of omega
    double* desc_part = nullptr; // learned start: descriptor terms per neighbour entry and atom
    double *e_nn_intra = nullptr, *e_nn_pair = nullptr;
    int* nmo = nullptr;
    // per-build data
    double *D = nullptr, *F = nullptr, *Jenv = nullptr, *omega = nullptr;
    double *tr_xy = nullptr, *tr_yx = nullptr, *trV = nullptr, *trJ = nullptr;
    double *E_int = nullptr, *E_scf = nullptr, *E_frag = nullptr, *E_tot = nullptr;
    // mixed precision: FP64 reference Hermite density and field of the last FP64 build
    double* Dh_ref[kClasses] = {};
    double* Jh_ref[kClasses] = {};
    bool have_ref = false;
    bool ref_exact = false;  // the reference field came from an FP64 build
    float* boys32 = nullptr;
    double* rec_resid = nullptr;  // workspace of the FP32-core records' charge-conserving rounding
    float* fc_qmin = nullptr;     // [n_frag*kClasses] smallest Schwarz factor per fragment and class
    int* iters = nullptr;
    int* err_flag = nullptr;
    double* diis = nullptr;
    int64_t diis_stride = 0;
    double* Jh[kClasses] = {};
    int njh[kClasses] = {};
    int2* tiles[kClasses][kClasses] = {};
    int n_tiles[kClasses * kClasses] = {};
    unsigned long long* qcount = nullptr;
    JPlanSet* jplan = nullptr;  // J-engine tile plans and work queues per engine
    // learned warm start
    double* rot = nullptr;
    double* Sh = nullptr;   // S^{1/2} per fragment (packed)
    double* Sih = nullptr;  // S^{-1/2} per fragment (packed)
    double* D_iso = nullptr;
    float* Xd = nullptr;
    float* Yd = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr, ev3 = nullptr;
};

}  // namespace fef

namespace fef {
static std::atomic<long long> g_launches{0};
void note_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace fef

using namespace fef;

static thread_local std::string g_create_error;  // message of the last failed context-free call

namespace fef {
void set_global_error(const char* msg) { g_create_error = msg; }
}  // namespace fef

#define FEF_API_BEGIN try {
#define FEF_API_END(ctx)                                              \
    }                                                                 \
    catch (const Error& e)                                            \
    {                                                                 \
        if (ctx) (ctx)->last_error = e.msg; else g_create_error = e.msg; \
        return e.status;                                              \
    }                                                                 \
    catch (const std::exception& e)                                   \
    {                                                                 \
        if (ctx) (ctx)->last_error = e.what(); else g_create_error = e.what(); \
        return FEF_ERR_ARG;                                           \
    }

static void require(bool ok, fef_status st, const std::string& msg)
{
    if (!ok) throw Error{st, msg};
}

extern "C" void fef_default_options(fef_options* o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = FEF_FP64;
    o->cutoff_A = 0.0;
    o->schwarz = 1e-12;
    o->e_tol = 1e-8;
    o->micro_e_tol = 1e-11;
    o->micro_comm_tol = 1e-9;
    o->max_macro = 100;
    o->max_micro = 200;
    o->diis_size = 8;
    o->start = FEF_START_SUPERPOSITION;
    o->use_graph = 1;
    o->mixed_switch = 1e-6;
    o->exact_engine = FEF_ENGINE_FP64;
    o->far_field = 0;
    o->mixed_build = FEF_MIXED_INCREMENT;
}

// ---------------------------------------------------------------------------------------------- helpers
static void check_device_flags(fef_ctx* c, const char* where)
{
    int flag = 0;
    ck(cudaMemcpyAsync(&flag, c->buf->err_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream), where);
    ck(cudaStreamSynchronize(c->stream), where);
    if (flag & kErrNumeric) throw Error{FEF_ERR_NUMERIC, std::string(where) + ": NaN/Inf in a matrix or energy"};
    if (flag & kErrBounds) throw Error{FEF_ERR_ARG, std::string(where) + ": device bounds check failed"};
}

static void clear_flags(fef_ctx* c)
{
    ck(cudaMemsetAsync(c->buf->err_flag, 0, sizeof(int), c->stream), "clear flags");
}

// One FEF Fock build from the context's current densities: Hermite densities, J-engine, back-transform,
// F = h + G + V_env + J_env, and all reference energies of the current densities.
//   fp32 = false: full FP64 J-engine; the Hermite density and field become the mixed-precision
//                 reference (D_ref, J[D_ref]).
//   fp32 = true : incremental J[D] = J[D_ref] + J_fp32[D - D_ref] (needs a reference).
// Kinds of Fock build.  FP64: the J-engine in FP64; its field becomes the exact reference.
// FP32_INC: J[D] = J[D_ref] + J_fp32[D - D_ref] with the stored reference (falls back to FP64 when
// there is none).  FP32_REF: the whole field from the FP32 core (D_ref = 0); it becomes an inexact
// reference, whose error is then the same for every later increment relative to it.
enum BuildKind { kBuildFP64 = 0, kBuildFP32Inc = 1, kBuildFP32Ref = 2 };

// Device timestamp (ns, %globaltimer) at this point of the stream: the per-phase timing inside a
// captured graph, where events cannot be timed.
__global__ void k_timestamp(unsigned long long* t)
{
    unsigned long long v;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
    *t = v;
}

// Phase marks: CUDA events when launching eagerly, device timestamps while capturing.
static void mark(fef_ctx* c, int i)
{
    Buffers* b = c->buf;
    if (b->capturing) {
        k_timestamp<<<1, 1, 0, c->stream>>>(b->stamps + i);
        note_launches(1);
        ck(cudaGetLastError(), "timestamp");
    } else {
        cudaEvent_t ev[4] = {b->ev0, b->ev1, b->ev2, b->ev3};
        ck(cudaEventRecord(ev[i], c->stream), "event");
    }
}

static void ensure_learn_buffers(fef_ctx* c);

// Intra-fragment ERI tasks (fragment, shell pair s1, shell pair s2 >= s1, first bra component; the task
// covers intra_nkb(la, lb, lc, ld) components) sorted by angular-momentum class
// cls = ((la 3 + lb) 3 + lc) 3 + ld; cls_off[c] = first task of class c.
static void intra_eri_tasks(int nf, const std::vector<int>& frag_sp0, const std::vector<int>& sp_a,
                            const std::vector<int>& sp_b, const std::vector<int>& sh_l, std::vector<int4>& tasks,
                            std::vector<int>& cls_off)
{
    std::vector<std::vector<int4>> by_cls(81);
    for (int x = 0; x < nf; ++x)
        for (int s1 = frag_sp0[x]; s1 < frag_sp0[x + 1]; ++s1)
            for (int s2 = s1; s2 < frag_sp0[x + 1]; ++s2) {
                const int la = sh_l[sp_a[s1]], lb = sh_l[sp_b[s1]], lc = sh_l[sp_a[s2]], ld = sh_l[sp_b[s2]];
                const int cls = ((la * 3 + lb) * 3 + lc) * 3 + ld;
                const int step = intra_nkb(la, lb, lc, ld);
                for (int k = 0; k < ncart(la) * ncart(lb); k += step) by_cls[cls].push_back(make_int4(x, s1, s2, k));
            }
    tasks.clear();
    cls_off.assign(82, 0);
    for (int c = 0; c < 81; ++c) {
        cls_off[c] = (int)tasks.size();
        tasks.insert(tasks.end(), by_cls[c].begin(), by_cls[c].end());
    }
    cls_off[81] = (int)tasks.size();
}

static int resolve_kind(const fef_ctx* c, int kind)
{
    return (kind == kBuildFP32Inc && !c->buf->have_ref) ? kBuildFP64 : kind;
}

// Device work of a build of a resolved kind (stream-ordered only, so that it can be captured).
static void build_fock_device(fef_ctx* c, int kind)
{
    Buffers* b = c->buf;
    const Dev& d = c->dev;
    cudaStream_t s = c->stream;
    const bool fp32 = kind != kBuildFP64;
    ck(launch_hermite_density(d, b->D, s), "hermite density");
    for (int L = 0; L < kClasses; ++L) {
        if (b->njh[L] == 0) continue;
        if (kind == kBuildFP32Inc)
            ck(cudaMemcpyAsync(b->Jh[L], b->Jh_ref[L], sizeof(double) * b->njh[L], cudaMemcpyDeviceToDevice, s), "Jh");
        else
            ck(cudaMemsetAsync(b->Jh[L], 0, sizeof(double) * b->njh[L], s), "zero Jh");
        if (kind == kBuildFP32Ref)
            ck(cudaMemsetAsync(b->Dh_ref[L], 0, sizeof(double) * b->njh[L], s), "zero reference");
    }
    if (fp32) ck(launch_fp32_records(d, b->Dh_ref, b->rec_resid, s), "fp32 records");
    const bool df = !fp32 && c->opt.exact_engine == FEF_ENGINE_DF64;
    if (df) ck(launch_df_density(d, s), "df64 density");
    const int2* tiles[kClasses][kClasses];
    for (int i = 0; i < kClasses; ++i)
        for (int j = 0; j < kClasses; ++j) tiles[i][j] = b->tiles[i][j];
    mark(c, 0);
    ck(jplan_launch(b->jplan, d, fp32 ? 1 : (df ? 2 : 0), tiles, b->n_tiles, c->opt.schwarz, s), "J-engine");
    mark(c, 1);
    if (kind != kBuildFP32Inc) {
        for (int L = 0; L < kClasses; ++L) {
            if (b->njh[L] == 0) continue;
            ck(cudaMemcpyAsync(b->Jh_ref[L], b->Jh[L], sizeof(double) * b->njh[L], cudaMemcpyDeviceToDevice, s), "ref");
            ck(cudaMemcpyAsync(b->Dh_ref[L], d.pp_Dh[L], sizeof(double) * b->njh[L], cudaMemcpyDeviceToDevice, s),
               "ref");
        }
    }
    ck(launch_back_transform(d, b->Jenv, s), "back-transform");
    ck(launch_fock_energy(d, b->h, b->Venv, b->Jenv, b->eric, b->D, b->F, b->omega, b->e_nn_intra, b->E_int,
                          b->trV, b->trJ, s),
       "fock");
    if (b->far_on)
        ck(launch_far_field(d, b->far_M, b->far_Mnuc, b->far_cen, b->D, b->far_mult, b->far_pot, b->far_E, b->F,
                            b->omega, s),
           "far field");
    ck(launch_nuclear_traces(d, b->trf_off, b->trf, b->tr_xy, b->tr_yx, s), "nuclear traces");
    ck(launch_energies(d, b->E_int, b->trV, b->trJ, b->tr_xy, b->tr_yx, b->e_nn_pair, b->E_frag, b->E_tot, s),
       "energies");
    if (b->far_on) ck(launch_far_energy(d, b->far_E, b->E_frag, b->E_tot, s), "far-field energies");
    ck(launch_check_finite(b->F, c->mat_total, b->err_flag, s), "check");
}

// Host-side state after a build of a resolved kind.
static void build_fock_host(fef_ctx* c, int kind)
{
    if (kind != kBuildFP32Inc) {
        c->buf->have_ref = true;
        c->buf->ref_exact = kind == kBuildFP64;
    }
    c->last_build_fp32 = kind != kBuildFP64;
    c->energies_valid = true;
}

static void build_fock_internal(fef_ctx* c, int kind = kBuildFP64)
{
    kind = resolve_kind(c, kind);
    build_fock_device(c, kind);
    build_fock_host(c, kind);
}

static void run_scf(fef_ctx* c, bool with_field, bool have_start)
{
    Buffers* b = c->buf;
    ScfArgs a{};
    a.h = b->h;
    a.omega = with_field ? b->omega : nullptr;
    a.S = b->S;
    a.X = b->X;
    a.nmo = b->nmo;
    a.eric = b->eric;
    a.eric_packed = 1;
    a.e_nn = b->e_nn_intra;
    a.D = b->D;
    a.F = b->F;
    a.diis_F = b->diis;
    a.diis_stride = b->diis_stride;
    a.E_scf = b->E_scf;
    a.E_int = b->E_int;
    a.iters = b->iters;
    a.have_start = have_start ? 1 : 0;
    a.max_iter = c->opt.max_micro;
    a.diis_size = c->opt.diis_size;
    a.e_tol = c->opt.micro_e_tol;
    a.comm_tol = c->opt.micro_comm_tol;
    a.ws = b->scf_ws;
    a.gap = b->gap;
    a.tol = b->scf_tol;
    a.shift_after = kScfShiftAfter;
    a.level_shift = kScfLevelShift;
    if (b->n_scf_big > 0) {
        a.list = b->scf_small;
        a.n_list = b->n_scf_small;
        a.big_list = b->scf_big;
        a.n_big = b->n_scf_big;
    }
    a.diis_by_moff = 1;
    mark(c, 2);
    ck(launch_fragment_scf(c->dev, a, c->max_nao, c->stream), "fragment SCF");
    mark(c, 3);
    c->energies_valid = false;
}

// micro-iteration counts of the last fragment SCF launch (negative = not converged) and its time
static void scf_counts(fef_ctx* c, double& max_it, double& sum_it, double& ms)
{
    std::vector<int> it(c->n_frag);
    ck(cudaMemcpyAsync(it.data(), c->buf->iters, sizeof(int) * c->n_frag, cudaMemcpyDeviceToHost, c->stream), "iters");
    ck(cudaStreamSynchronize(c->stream), "iters");
    max_it = 0;
    sum_it = 0;
    for (int v : it) {
        max_it = std::max<double>(max_it, std::abs(v));
        sum_it += std::abs(v);
    }
    float f = 0.f;
    ck(cudaEventElapsedTime(&f, c->buf->ev2, c->buf->ev3), "event time");
    ms = f;
}

// Micro-iteration thresholds of the next fragment SCF (stream-ordered copy from pinned memory, made
// before a graph replay so that captured graphs read them from device memory).  progress: the
// energy change of the previous macro-iteration (< 0: the options' thresholds).  An SCF in a field
// that will still move by ~progress need not be converged below ~1e-3 progress (commutator) and
// ~1e-5 progress (energy); the options' thresholds are the floor, so the last macro-iterations and
// the fixed point are those of tightly converged fragment SCFs.
static void set_scf_thresholds(fef_ctx* c, double progress)
{
    Buffers* b = c->buf;
    const fef_options& o = c->opt;
    double e = o.micro_e_tol, m = o.micro_comm_tol;
    if (progress >= 0.0) {
        e = std::max(o.micro_e_tol, std::min(1e-7, 1e-5 * progress));
        m = std::max(o.micro_comm_tol, std::min(1e-5, 1e-3 * progress));
    }
    if (e == b->scf_tol_host[0] && m == b->scf_tol_host[1]) return;
    ck(cudaStreamSynchronize(c->stream), "thresholds");  // the previous copy has been consumed
    b->scf_tol_host[0] = e;
    b->scf_tol_host[1] = m;
    ck(cudaMemcpyAsync(b->scf_tol, b->scf_tol_host, 2 * sizeof(double), cudaMemcpyHostToDevice, c->stream),
       "thresholds");
}

// ------------------------------------------------------------------------------ one macro-iteration
// Pinned read-back layout: E_tot at 0, error flag at 8, E_frag[n] at 16, iters[n] after E_frag.
static double* stage_Et(fef_ctx* c) { return reinterpret_cast<double*>(c->buf->stage); }
static int* stage_flag(fef_ctx* c) { return reinterpret_cast<int*>(c->buf->stage + 8); }
static double* stage_Ex(fef_ctx* c) { return reinterpret_cast<double*>(c->buf->stage + 16); }
static int* stage_iters(fef_ctx* c) { return reinterpret_cast<int*>(c->buf->stage + 16 + 8 * (size_t)c->n_frag); }
static unsigned long long* stage_stamps(fef_ctx* c)
{
    return reinterpret_cast<unsigned long long*>(c->buf->stage + 16 + 16 * (size_t)c->n_frag);
}

// Device work of macro-iteration k >= 1: every fragment's RHF in the field omega^(k) (from D^(k-1)),
// then the Fock build of the kind given from D^(k), then the read-back of the energies, the
// micro-iteration counts and the error flag into pinned memory.  Stream-ordered only.
static void macro_step_device(fef_ctx* c, int kind)
{
    Buffers* b = c->buf;
    cudaStream_t s = c->stream;
    run_scf(c, true, true);
    build_fock_device(c, kind);
    ck(cudaMemcpyAsync(stage_Et(c), b->E_tot, sizeof(double), cudaMemcpyDeviceToHost, s), "read-back");
    ck(cudaMemcpyAsync(stage_flag(c), b->err_flag, sizeof(int), cudaMemcpyDeviceToHost, s), "read-back");
    ck(cudaMemcpyAsync(stage_Ex(c), b->E_frag, sizeof(double) * c->n_frag, cudaMemcpyDeviceToHost, s), "read-back");
    ck(cudaMemcpyAsync(stage_iters(c), b->iters, sizeof(int) * c->n_frag, cudaMemcpyDeviceToHost, s), "read-back");
    if (b->capturing)
        ck(cudaMemcpyAsync(stage_stamps(c), b->stamps, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s),
           "read-back");
}

// One macro-iteration: with opt.use_graph, replay the CUDA graph of this kind (captured on first
// use: one graph launch instead of ~30 kernel launches and copies); then one synchronisation.
static void macro_step(fef_ctx* c, int kind)
{
    Buffers* b = c->buf;
    if (c->opt.use_graph) {
        if (!b->macro_graph[kind]) {
            // captured on a private non-blocking stream (the legacy default stream cannot be
            // captured), replayed on the context stream
            if (!b->capture_stream)
                ck(cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking), "capture stream");
            ck(cudaStreamSynchronize(c->stream), "graph capture");
            const long long l0 = launches_so_far();
            cudaGraph_t g = nullptr;
            const cudaStream_t user = c->stream;
            c->stream = b->capture_stream;
            b->capturing = true;
            // relaxed: the launchers set kernel attributes (cudaFuncSetAttribute) while capturing
            cudaError_t e0 = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed);
            if (e0 != cudaSuccess) {
                c->stream = user;
                b->capturing = false;
            }
            ck(e0, "graph capture");
            try {
                macro_step_device(c, kind);
            } catch (...) {
                cudaStreamEndCapture(c->stream, &g);
                if (g) cudaGraphDestroy(g);
                c->stream = user;
                b->capturing = false;
                throw;
            }
            const cudaError_t e1 = cudaStreamEndCapture(c->stream, &g);
            c->stream = user;
            b->capturing = false;
            ck(e1, "graph capture");
            const cudaError_t e = cudaGraphInstantiate(&b->macro_graph[kind], g, 0);
            cudaGraphDestroy(g);
            ck(e, "graph instantiate");
            b->macro_graph_launches[kind] = launches_so_far() - l0;
            note_launches(-b->macro_graph_launches[kind]);  // nothing ran during the capture
        }
        ck(cudaGraphLaunch(b->macro_graph[kind], c->stream), "graph launch");
        note_launches(b->macro_graph_launches[kind]);
    } else {
        macro_step_device(c, kind);
    }
    ck(cudaStreamSynchronize(c->stream), "macro-iteration");
}

// ---------------------------------------------------------------------------------------------- create
extern "C" fef_status fef_create(const fef_geometry* g, const fef_basis* bs, const fef_options* opt,
                                 void* cuda_stream, fef_ctx** out)
{
    fef_ctx* c = nullptr;
    try {
        require(g && bs && out, FEF_ERR_ARG, "fef_create: NULL geometry, basis or output pointer");
        *out = nullptr;
        require(g->n_atoms > 0 && g->n_frag > 0 && g->Z && g->xyz && g->frag_of_atom && g->basis_of_atom,
                FEF_ERR_ARG, "fef_create: empty geometry or NULL geometry arrays");
        require(bs->n_sets > 0 && bs->set_shell_offset && bs->shell_l && bs->shell_nprim && bs->exps && bs->coefs,
                FEF_ERR_ARG, "fef_create: empty basis or NULL basis arrays");
        c = new fef_ctx();
        if (opt) c->opt = *opt; else fef_default_options(&c->opt);
        const fef_options& o = c->opt;
        require(o.diis_size >= 1 && o.diis_size <= 8, FEF_ERR_ARG, "options: diis_size must be 1..8");
        require(o.max_macro >= 1 && o.max_micro >= 1, FEF_ERR_ARG, "options: iteration limits must be >= 1");
        require(o.precision == FEF_FP64 || o.precision == FEF_MIXED, FEF_ERR_ARG, "options: bad precision");
        require(o.far_field == 0 || o.far_field == 1, FEF_ERR_ARG, "options: far_field must be 0 or 1");
        require(o.exact_engine == FEF_ENGINE_FP64 || o.exact_engine == FEF_ENGINE_DF64, FEF_ERR_ARG,
                "options: bad exact_engine");
        require(o.schwarz >= 0.0 && std::isfinite(o.schwarz), FEF_ERR_ARG, "options: bad schwarz threshold");
        require(!std::isnan(o.cutoff_A), FEF_ERR_ARG, "options: cutoff_A is NaN");
        require(o.e_tol > 0.0 && std::isfinite(o.e_tol), FEF_ERR_ARG, "options: e_tol must be finite and > 0");
        require(o.micro_e_tol > 0.0 && std::isfinite(o.micro_e_tol) && o.micro_comm_tol > 0.0 &&
                    std::isfinite(o.micro_comm_tol),
                FEF_ERR_ARG, "options: micro_e_tol and micro_comm_tol must be finite and > 0");
        require(o.mixed_switch >= 0.0 && std::isfinite(o.mixed_switch), FEF_ERR_ARG, "options: bad mixed_switch");
        require(o.mixed_build == FEF_MIXED_INCREMENT || o.mixed_build == FEF_MIXED_WHOLE, FEF_ERR_ARG,
                "options: bad mixed_build");
        c->stream = static_cast<cudaStream_t>(cuda_stream);

        const int na = g->n_atoms, nf = g->n_frag;
        c->n_atoms = na;
        c->n_frag = nf;
        // ---- fragments: contiguous runs in order
        std::vector<int> frag_atom0(nf, -1), frag_nat(nf, 0);
        for (int a = 0; a < na; ++a) {
            int x = g->frag_of_atom[a];
            require(x >= 0 && x < nf, FEF_ERR_GEOM, "frag_of_atom out of range");
            require(a == 0 ? x == 0 : (x == g->frag_of_atom[a - 1] || x == g->frag_of_atom[a - 1] + 1),
                    FEF_ERR_GEOM, "fragments must be contiguous atom runs numbered in order");
            if (frag_atom0[x] < 0) frag_atom0[x] = a;
            frag_nat[x]++;
        }
        require(g->frag_of_atom[na - 1] == nf - 1, FEF_ERR_GEOM, "n_frag does not match frag_of_atom");
        for (int a = 0; a < na; ++a) {
            require(g->Z[a] >= 1 && g->Z[a] <= 36, FEF_ERR_GEOM, "nuclear charge out of range 1..36");
            for (int k = 0; k < 3; ++k) require(std::isfinite(g->xyz[3 * a + k]), FEF_ERR_GEOM, "non-finite coordinate");
            require(g->basis_of_atom[a] >= 0 && g->basis_of_atom[a] < bs->n_sets, FEF_ERR_ARG,
                    "basis_of_atom out of range");
        }
        // coincident atoms inside a fragment
        for (int x = 0; x < nf; ++x)
            for (int a = frag_atom0[x]; a < frag_atom0[x] + frag_nat[x]; ++a)
                for (int b2 = frag_atom0[x]; b2 < a; ++b2) {
                    double r2 = 0;
                    for (int k = 0; k < 3; ++k) r2 += std::pow(g->xyz[3 * a + k] - g->xyz[3 * b2 + k], 2);
                    require(r2 > 1e-6, FEF_ERR_GEOM, "coincident atoms in fragment " + std::to_string(x));
                }
        // ---- basis sets
        int n_shell_types = bs->set_shell_offset[bs->n_sets];
        require(bs->set_shell_offset[0] == 0 && n_shell_types > 0, FEF_ERR_BASIS, "bad set_shell_offset");
        std::vector<int> type_p0(n_shell_types + 1, 0);
        for (int k = 0; k < n_shell_types; ++k) {
            require(bs->shell_l[k] >= 0 && bs->shell_l[k] <= kMaxL, FEF_ERR_BASIS, "shell l must be 0, 1 or 2");
            require(bs->shell_nprim[k] >= 1 && bs->shell_nprim[k] <= 8, FEF_ERR_BASIS, "shell nprim must be 1..8");
            type_p0[k + 1] = type_p0[k] + bs->shell_nprim[k];
        }
        for (int i = 0; i < type_p0[n_shell_types]; ++i) {
            require(std::isfinite(bs->exps[i]) && bs->exps[i] > 0.0, FEF_ERR_BASIS, "exponents must be positive");
            require(std::isfinite(bs->coefs[i]), FEF_ERR_BASIS, "non-finite contraction coefficient");
        }
        for (int k = 0; k < bs->n_sets; ++k)
            require(bs->set_shell_offset[k + 1] >= bs->set_shell_offset[k], FEF_ERR_BASIS, "bad set_shell_offset");
        // ---- shells, prims, AOs
        std::vector<int> sh_l, sh_np, sh_p0, sh_ao, sh_atom, p_l;
        std::vector<double> p_exp, p_coef_raw;
        std::vector<int> frag_sh0(nf), frag_nsh(nf), frag_nao(nf), frag_ao0(nf), frag_nocc(nf);
        std::vector<int> ao_sh, ao_k;
        int max_l = 0;
        int ao_global = 0;
        for (int x = 0; x < nf; ++x) {
            frag_sh0[x] = (int)sh_l.size();
            frag_ao0[x] = ao_global;
            int ao = 0, ne = 0;
            for (int a = frag_atom0[x]; a < frag_atom0[x] + frag_nat[x]; ++a) {
                ne += g->Z[a];
                int set = g->basis_of_atom[a];
                for (int k = bs->set_shell_offset[set]; k < bs->set_shell_offset[set + 1]; ++k) {
                    int l = bs->shell_l[k];
                    max_l = std::max(max_l, l);
                    int sid = (int)sh_l.size();
                    sh_l.push_back(l);
                    sh_np.push_back(bs->shell_nprim[k]);
                    sh_p0.push_back((int)p_exp.size());
                    sh_ao.push_back(ao);
                    sh_atom.push_back(a);
                    for (int i = 0; i < bs->shell_nprim[k]; ++i) {
                        p_exp.push_back(bs->exps[type_p0[k] + i]);
                        p_coef_raw.push_back(bs->coefs[type_p0[k] + i]);
                        p_l.push_back(l);
                    }
                    for (int q = 0; q < ncart(l); ++q) {
                        ao_sh.push_back(sid);
                        ao_k.push_back(q);
                    }
                    ao += ncart(l);
                }
            }
            frag_nsh[x] = (int)sh_l.size() - frag_sh0[x];
            require(ao > 0, FEF_ERR_BASIS, "fragment " + std::to_string(x) + " has no basis functions");
            frag_nao[x] = ao;
            ao_global += ao;
            ne -= g->charge ? g->charge[x] : 0;
            require(ne >= 0 && ne % 2 == 0, FEF_ERR_GEOM,
                    "fragment " + std::to_string(x) + " needs an even, non-negative electron count");
            frag_nocc[x] = ne / 2;
        }
        c->n_shells = (int)sh_l.size();
        c->n_prims = (int)p_exp.size();
        int max_nao = *std::max_element(frag_nao.begin(), frag_nao.end());
        require(max_nao <= kMaxFragAO, FEF_ERR_ARG,
                "fragments above " + std::to_string(kMaxFragAO) + " AOs are not supported");
        c->max_nao = max_nao;
        c->nao = frag_nao;
        c->nocc = frag_nocc;
        std::vector<int64_t> moff(nf + 1, 0), eoff(nf + 1, 0), coff(nf + 1, 0);
        for (int x = 0; x < nf; ++x) {
            int64_t n = frag_nao[x], np = n * (n + 1) / 2;
            moff[x + 1] = moff[x] + n * n;
            eoff[x + 1] = eoff[x] + n * n * n * n;
            coff[x + 1] = coff[x] + np * np;
        }
        c->coff_total = coff[nf];
        c->moff = moff;
        c->mat_total = moff[nf];
        c->eri_total = eoff[nf];
        // ---- shell pairs and primitive pairs (class-sorted)
        std::vector<int> sp_a, sp_b, sp_L, frag_sp0(nf + 1, 0);
        for (int x = 0; x < nf; ++x) {
            frag_sp0[x] = (int)sp_a.size();
            for (int a = 0; a < frag_nsh[x]; ++a)
                for (int b2 = a; b2 < frag_nsh[x]; ++b2) {
                    int s1 = frag_sh0[x] + a, s2 = frag_sh0[x] + b2;
                    sp_a.push_back(s1);
                    sp_b.push_back(s2);
                    sp_L.push_back(sh_l[s1] + sh_l[s2]);
                }
        }
        frag_sp0[nf] = (int)sp_a.size();
        c->n_sp = (int)sp_a.size();
        std::vector<int> sp_pp0(c->n_sp, 0), frag_pp0(nf * kClasses), frag_npp(nf * kClasses);
        std::vector<int> pp_sp[kClasses], pp_ij[kClasses];
        for (int L = 0; L < kClasses; ++L)
            for (int x = 0; x < nf; ++x) {
                frag_pp0[x * kClasses + L] = (int)pp_sp[L].size();
                for (int sp = frag_sp0[x]; sp < frag_sp0[x + 1]; ++sp) {
                    if (sp_L[sp] != L) continue;
                    sp_pp0[sp] = (int)pp_sp[L].size();
                    for (int i = 0; i < sh_np[sp_a[sp]]; ++i)
                        for (int j = 0; j < sh_np[sp_b[sp]]; ++j) {
                            pp_sp[L].push_back(sp);
                            pp_ij[L].push_back(i * 16 + j);
                        }
                }
                frag_npp[x * kClasses + L] = (int)pp_sp[L].size() - frag_pp0[x * kClasses + L];
            }
        // J-engine bra order: inside each fragment's class range, primitive pairs by increasing exponent
        // p = a + b, so that a warp's 32 bra pairs are of similar extent and take the same Boys branch
        std::vector<int> pp_perm[kClasses];
        for (int L = 0; L < kClasses; ++L) {
            const int n = (int)pp_sp[L].size();
            std::vector<double> pexp(n);
            for (int g2 = 0; g2 < n; ++g2) {
                const int sp = pp_sp[L][g2], ij = pp_ij[L][g2];
                pexp[g2] = p_exp[sh_p0[sp_a[sp]] + (ij >> 4)] + p_exp[sh_p0[sp_b[sp]] + (ij & 15)];
            }
            pp_perm[L].resize(n);
            for (int g2 = 0; g2 < n; ++g2) pp_perm[L][g2] = g2;
            for (int x = 0; x < nf; ++x) {
                auto first = pp_perm[L].begin() + frag_pp0[x * kClasses + L];
                std::stable_sort(first, first + frag_npp[x * kClasses + L],
                                 [&](int u, int v) { return pexp[u] < pexp[v]; });
            }
        }

        // ---- device upload
        ck(cudaGetDevice(&c->device), "cudaGetDevice");  // every host-side check comes before this
        c->buf = new Buffers();
        Buffers* b = c->buf;
        cudaStream_t s = c->stream;
        b->pool = device_pool(c->device);
        b->as = s;
        Dev& d = c->dev;
        d.n_frag = nf;
        d.n_atoms = na;
        d.n_shells = c->n_shells;
        d.n_sp = c->n_sp;
        d.max_nao = max_nao;
        d.max_l = max_l;
        std::vector<double> xyzA(g->xyz, g->xyz + 3 * na), Zd(na);
        for (int a = 0; a < na; ++a) Zd[a] = g->Z[a];
        double* xyz_A = b->upload(xyzA, s, "xyz");
        double* atom_xyz = b->alloc<double>(3 * na, "atom_xyz");
        d.atom_xyz = atom_xyz;
        d.atom_Z = b->upload(Zd, s, "Z");
        d.frag_atom0 = b->upload(frag_atom0, s, "frag");
        d.frag_nat = b->upload(frag_nat, s, "frag");
        d.frag_sh0 = b->upload(frag_sh0, s, "frag");
        d.frag_nsh = b->upload(frag_nsh, s, "frag");
        d.frag_nao = b->upload(frag_nao, s, "frag");
        d.frag_ao0 = b->upload(frag_ao0, s, "frag");
        d.frag_sp0 = b->upload(frag_sp0, s, "frag");
        d.frag_nocc = b->upload(frag_nocc, s, "frag");
        d.frag_moff = b->upload(moff, s, "frag");
        d.frag_eoff = b->upload(eoff, s, "frag");
        d.frag_coff = b->upload(coff, s, "frag");
        d.frag_pp0 = b->upload(frag_pp0, s, "frag");
        d.frag_npp = b->upload(frag_npp, s, "frag");
        d.sh_l = b->upload(sh_l, s, "shells");
        d.sh_np = b->upload(sh_np, s, "shells");
        d.sh_p0 = b->upload(sh_p0, s, "shells");
        d.sh_ao = b->upload(sh_ao, s, "shells");
        d.sh_atom = b->upload(sh_atom, s, "shells");
        d.p_exp = b->upload(p_exp, s, "prims");
        double* p_coef_raw_d = b->upload(p_coef_raw, s, "prims");
        int* p_l_d = b->upload(p_l, s, "prims");
        double* p_coef = b->alloc<double>(p_exp.size(), "prims");
        d.p_coef = p_coef;
        d.ao_sh = b->upload(ao_sh, s, "aos");
        d.ao_k = b->upload(ao_k, s, "aos");
        double* ao_scale = b->alloc<double>(ao_global, "aos");
        d.ao_scale = ao_scale;
        d.sp_a = b->upload(sp_a, s, "shell pairs");
        d.sp_b = b->upload(sp_b, s, "shell pairs");
        d.sp_L = b->upload(sp_L, s, "shell pairs");
        d.sp_pp0 = b->upload(sp_pp0, s, "shell pairs");
        double* sp_Q = b->alloc<double>(c->n_sp, "shell pairs");
        d.sp_Q = sp_Q;
        double4_32a* ppP[kClasses];
        float4* ppPf[kClasses];
        float4* ppPr[kClasses];
        float4* ppPhi[kClasses];
        float4* ppPlo[kClasses];
        float2* ppSq[kClasses];
        double* ppK[kClasses];
        float* ppQ[kClasses];
        double* ppRp[kClasses];
        int max_npp = 1;
        for (int L = 0; L < kClasses; ++L) {
            int n = (int)pp_sp[L].size();
            d.n_pp[L] = n;
            d.pp_sp[L] = b->upload(pp_sp[L], s, "prim pairs");
            d.pp_ij[L] = b->upload(pp_ij[L], s, "prim pairs");
            ppP[L] = b->alloc<double4_32a>(n, "prim pairs");
            ppPf[L] = b->alloc<float4>(n, "prim pairs");
            ppPr[L] = b->alloc<float4>(n, "prim pairs");
            d.pp_Pr[L] = ppPr[L];
            d.pp_Dh32[L] = b->alloc<float>((size_t)nh(L) * n, "fp32 pair scratch");
            ppPhi[L] = b->alloc<float4>(n, "prim pairs df64");
            ppPlo[L] = b->alloc<float4>(n, "prim pairs df64");
            d.pp_Phi[L] = ppPhi[L];
            d.pp_Plo[L] = ppPlo[L];
            d.pp_udf[L] = b->alloc<float2>((size_t)nh(L) * n, "hermite weights df64");
            ppSq[L] = b->alloc<float2>(n, "prim pairs df64");
            d.pp_sqdf[L] = ppSq[L];
            b->Dh_ref[L] = b->alloc<double>((size_t)nh(L) * n, "hermite density ref");
            b->Jh_ref[L] = b->alloc<double>((size_t)nh(L) * n, "hermite field ref");
            ppK[L] = b->alloc<double>(n, "prim pairs");
            ppQ[L] = b->alloc<float>(n, "prim pairs");
            ppRp[L] = b->alloc<double>(n, "prim pairs");
            d.pp_rp[L] = ppRp[L];
            d.pp_perm[L] = b->upload(pp_perm[L], s, "prim pairs");
            d.pp_rec32[L] = b->alloc<float>((size_t)rec32_len(L) * n, "fp32 records");
            max_npp = std::max(max_npp, n);
            d.pp_P[L] = ppP[L];
            d.pp_Pf[L] = ppPf[L];
            d.pp_K[L] = ppK[L];
            d.pp_Q[L] = ppQ[L];
            b->njh[L] = nh(L) * n;
            d.pp_Dh[L] = b->alloc<double>((size_t)nh(L) * n, "hermite density");
            d.pp_u[L] = b->alloc<double>((size_t)nh(L) * n, "hermite weights");
            b->Jh[L] = b->alloc<double>((size_t)nh(L) * n, "hermite field");
            d.pp_Jh[L] = b->Jh[L];
            // pool memory comes back with old contents: the per-build inputs start as zeros (no
            // reference density; FP32 records of zero weight) until a build or fef_autotune fills them
            const size_t nhn = (size_t)nh(L) * n;
            ck(cudaMemsetAsync(b->Dh_ref[L], 0, sizeof(double) * nhn, s), "zero");
            ck(cudaMemsetAsync(d.pp_Dh[L], 0, sizeof(double) * nhn, s), "zero");
            ck(cudaMemsetAsync(d.pp_u[L], 0, sizeof(double) * nhn, s), "zero");
            ck(cudaMemsetAsync(d.pp_Dh32[L], 0, sizeof(float) * nhn, s), "zero");
            ck(cudaMemsetAsync(d.pp_udf[L], 0, sizeof(float2) * nhn, s), "zero");
            ck(cudaMemsetAsync(d.pp_rec32[L], 0, sizeof(float) * rec32_len(L) * (size_t)n, s), "zero");
        }
        b->rec_resid = b->alloc<double>(max_npp, "fp32 record residues");
        b->fc_qmin = b->alloc<float>((size_t)nf * kClasses, "class Schwarz minimum");
        d.fc_qmin = b->fc_qmin;
        b->boys = b->alloc<double>((size_t)kBoysRows * kBoysRowLen, "boys");
        d.boys = b->boys;
        b->boys32 = b->alloc<float>((size_t)kBoys32Rows * kBoysRowLen, "boys32");
        d.boys32 = b->boys32;
        float2* boysdf = b->alloc<float2>((size_t)kBoysRows * kBoysRowLen, "boys df64");
        d.boysdf = boysdf;
        b->err_flag = b->alloc<int>(1, "flag");
        d.err_flag = b->err_flag;
        ck(cudaMemsetAsync(b->err_flag, 0, sizeof(int), s), "flag");
        ck(cudaEventCreate(&b->ev0), "event");
        ck(cudaEventCreate(&b->ev1), "event");
        ck(cudaEventCreate(&b->ev2), "event");
        ck(cudaEventCreate(&b->ev3), "event");

        // ---- geometry-time kernels
        ck(launch_prepare(d, xyz_A, atom_xyz, p_coef, p_coef_raw_d, p_l_d, c->n_prims, s), "prepare");
        ck(launch_boys_table(b->boys, s), "boys table");
        ck(launch_boys_table32(b->boys, b->boys32, s), "boys table fp32");
        ck(launch_ao_scale(d, ao_scale, ao_global, nullptr, s), "ao scale");
        ck(launch_prim_pairs(d, ppP, ppPf, ppK, ppPr, ppRp, s), "prim pairs");
        ck(launch_df_setup(d, ppPhi, ppPlo, ppSq, boysdf, s), "df64 pair data");
        b->S = b->alloc<double>(c->mat_total, "S");
        b->h = b->alloc<double>(c->mat_total, "h");
        ck(launch_one_electron(d, b->S, b->h, s), "one-electron");
        // the learned warm start needs fragments of one kind (same atoms and s/p basis)
        bool learn_ok = true;
        for (int x = 1; x < nf && learn_ok; ++x) learn_ok = frag_nat[x] == frag_nat[0] && frag_nao[x] == frag_nao[0];
        learn_ok = learn_ok && max_l <= 1;
        if (learn_ok) {
            c->learn_desc = 4 * frag_nat[0];
            c->learn_pack = frag_nao[0] * (frag_nao[0] + 1) / 2;
            c->learn_feat = c->learn_desc + c->learn_pack;  // + the multipole estimate of omega
        }
        b->far_on = o.far_field && o.cutoff_A > 0.0;
        if (b->far_on || learn_ok) {
            // centroids of nuclear charge and nuclear moments (bohr), moment integrals about them
            std::vector<double> cen(3 * (size_t)nf, 0.0), mnuc(10 * (size_t)nf, 0.0);
            for (int x = 0; x < nf; ++x) {
                double zs = 0.0;
                for (int a = frag_atom0[x]; a < frag_atom0[x] + frag_nat[x]; ++a) {
                    zs += g->Z[a];
                    for (int k = 0; k < 3; ++k) cen[3 * x + k] += g->Z[a] * g->xyz[3 * a + k] / 0.529177210903;
                }
                for (int k = 0; k < 3; ++k) cen[3 * x + k] /= zs;
                for (int a = frag_atom0[x]; a < frag_atom0[x] + frag_nat[x]; ++a) {
                    double r[3];
                    for (int k = 0; k < 3; ++k) r[k] = g->xyz[3 * a + k] / 0.529177210903 - cen[3 * x + k];
                    const double z = g->Z[a];
                    const double v[10] = {z, z * r[0], z * r[1], z * r[2], z * r[0] * r[0], z * r[0] * r[1],
                                          z * r[0] * r[2], z * r[1] * r[1], z * r[1] * r[2], z * r[2] * r[2]};
                    for (int k = 0; k < 10; ++k) mnuc[10 * x + k] += v[k];
                }
            }
            b->far_cen = b->upload(cen, s, "far field");
            b->far_Mnuc = b->upload(mnuc, s, "far field");
            b->far_M = b->alloc<double>(10 * c->mat_total, "moment integrals");
            b->far_mult = b->alloc<double>(10 * (size_t)nf, "far field");
            b->far_pot = b->alloc<double>(10 * (size_t)nf, "far field");
            b->far_E = b->alloc<double>(nf, "far field");
            ck(launch_moment_integrals(d, b->far_cen, b->far_M, s), "moment integrals");
        }
        b->rot = b->alloc<double>((size_t)9 * nf, "frames");
        ck(launch_frames(d, b->rot, s), "frames");
        // neighbour list (within the cutoff) -> pairs x<y and CSR
        std::vector<unsigned char> flags((size_t)nf * nf, 0);
        {
            unsigned char* fl = b->alloc<unsigned char>((size_t)nf * nf, "neighbour flags");
            ck(cudaMemsetAsync(fl, 0, (size_t)nf * nf, s), "neighbour flags");
            double cutoff_bohr = o.cutoff_A > 0 ? o.cutoff_A / 0.529177210903 : 0.0;
            ck(launch_neighbours(d, cutoff_bohr, fl, s), "neighbours");
            ck(cudaMemcpyAsync(flags.data(), fl, flags.size(), cudaMemcpyDeviceToHost, s), "neighbours");
            ck(cudaStreamSynchronize(s), "neighbours");
            b->release(fl);
        }
        std::vector<int> pair_x, pair_y, nbr0(nf + 1, 0), nbr, nbr_pair;
        std::vector<std::vector<int>> adj(nf), adjp(nf);
        for (int x = 0; x < nf; ++x)
            for (int y = x + 1; y < nf; ++y)
                if (flags[(size_t)x * nf + y]) {
                    int p = (int)pair_x.size();
                    pair_x.push_back(x);
                    pair_y.push_back(y);
                    adj[x].push_back(y);
                    adjp[x].push_back(p);
                    adj[y].push_back(x);
                    adjp[y].push_back(p);
                }
        for (int x = 0; x < nf; ++x) {
            nbr0[x + 1] = nbr0[x] + (int)adj[x].size();
            // neighbours in ascending fragment order
            std::vector<int> idx(adj[x].size());
            for (size_t k = 0; k < idx.size(); ++k) idx[k] = (int)k;
            std::sort(idx.begin(), idx.end(), [&](int i, int j) { return adj[x][i] < adj[x][j]; });
            for (int k : idx) {
                nbr.push_back(adj[x][k]);
                nbr_pair.push_back(adjp[x][k]);
            }
        }
        c->n_pairs = (int)pair_x.size();
        d.n_pairs = c->n_pairs;
        c->h_pair_x = pair_x;
        c->h_pair_y = pair_y;
        c->h_frag_sp0 = frag_sp0;
        c->h_sp_a = sp_a;
        c->h_sp_b = sp_b;
        c->h_sh_l = sh_l;
        c->h_frag_pp0 = frag_pp0;
        c->h_frag_npp = frag_npp;
        d.pair_x = b->upload(pair_x, s, "pairs");
        d.pair_y = b->upload(pair_y, s, "pairs");
        d.frag_nbr0 = b->upload(nbr0, s, "pairs");
        d.nbr = b->upload(nbr, s, "pairs");
        c->n_nbr = (int)nbr.size();
        if (c->learn_feat > 0) ensure_learn_buffers(c);  // no allocation inside fef_iterate's learned start
        d.nbr_pair = b->upload(nbr_pair, s, "pairs");
        b->e_nn_intra = b->alloc<double>(nf, "e_nn");
        b->e_nn_pair = b->alloc<double>(c->n_pairs, "e_nn");
        ck(launch_nuclear_repulsion(d, b->e_nn_intra, b->e_nn_pair, s), "nuclear repulsion");
        // intra-fragment two-electron tensor -> Schwarz factors and C = (mu nu|ls) - (mu l|nu s)/2
        {
            double* eri = b->alloc<double>(c->coff_total, "intra eri");  // pair-packed U[pq][rs]
            // tasks: (fragment, shell pair s1 <= s2, bra component), sorted by class
            std::vector<int4> tasks;
            std::vector<int> cls_off;
            intra_eri_tasks(nf, frag_sp0, sp_a, sp_b, sh_l, tasks, cls_off);
            int4* tasks_d = b->upload(tasks, s, "intra tasks");
            ck(launch_intra_eri(d, tasks_d, cls_off, eri, s), "intra eri");
            ck(launch_schwarz(d, eri, sp_Q, ppQ, s), "schwarz");
            ck(launch_class_qmin(d, b->fc_qmin, s), "class Schwarz minimum");
            b->eric = b->alloc<double>(c->coff_total, "eric");
            ck(launch_coulomb_exchange(d, eri, b->eric, s), "coulomb-exchange");
            ck(cudaStreamSynchronize(s), "intra eri");
            b->release(eri);
            b->release(tasks_d);
        }
        b->Venv = b->alloc<double>(c->mat_total, "Venv");
        {
            double* vh[kClasses];
            for (int L = 0; L < kClasses; ++L) vh[L] = b->alloc<double>((size_t)nh(L) * d.n_pp[L], "Vh");
            ck(launch_nuclear_env(d, vh, b->Venv, s), "nuclear env");
            ck(cudaStreamSynchronize(s), "nuclear env");
            for (int L = 0; L < kClasses; ++L) b->release(vh[L]);
        }
        b->X = b->alloc<double>(c->mat_total, "X");
        b->nmo = b->alloc<int>(nf, "nmo");
        b->Sh = b->alloc<double>(c->mat_total, "S^1/2");
        b->Sih = b->alloc<double>(c->mat_total, "S^-1/2");
        double* orth_ws = max_nao > kOrthSmemMaxN ? b->alloc<double>(2 * c->mat_total, "orthogonaliser workspace")
                                                  : nullptr;
        ck(launch_orthogonaliser(d, b->S, b->X, b->nmo, 1e-7, max_nao, s, b->Sh, b->Sih, orth_ws), "orthogonaliser");
        c->nmo.assign(nf, 0);
        ck(cudaMemcpyAsync(c->nmo.data(), b->nmo, sizeof(int) * nf, cudaMemcpyDeviceToHost, s), "nmo");
        ck(cudaStreamSynchronize(s), "create");
        if (orth_ws) b->release(orth_ws);
        for (int x = 0; x < nf; ++x)
            require(c->nmo[x] >= frag_nocc[x], FEF_ERR_BASIS,
                    "fragment " + std::to_string(x) + ": basis too linearly dependent for its electrons");
        // J-engine tiles: (2*pair + swap, first of 32 bra primitive pairs).  For a pair (x, y) and
        // classes (Lx, Ly) the member with the larger class is the bra (lane-owned, no reduction);
        // swap = 1 when that is y.  Kernels with L_bra < L_ket are never needed.
        int64_t prim_q = 0;
        std::vector<int2> tl[kClasses][kClasses];
        for (int p = 0; p < c->n_pairs; ++p)
            for (int Lx = 0; Lx < kClasses; ++Lx)
                for (int Ly = 0; Ly < kClasses; ++Ly) {
                    const bool swap = Lx < Ly;
                    const int bx = swap ? pair_y[p] : pair_x[p], ky = swap ? pair_x[p] : pair_y[p];
                    const int LP = swap ? Ly : Lx, LQ = swap ? Lx : Ly;
                    int nb = frag_npp[bx * kClasses + LP], nk = frag_npp[ky * kClasses + LQ];
                    if (nb == 0 || nk == 0) continue;
                    for (int o2 = 0; o2 < nb; o2 += 32) {
                        tl[LP][LQ].push_back(make_int2(2 * p + (swap ? 1 : 0), frag_pp0[bx * kClasses + LP] + o2));
                        prim_q += (int64_t)std::min(32, nb - o2) * nk;
                    }
                }
        for (int LP = 0; LP < kClasses; ++LP)
            for (int LQ = 0; LQ < kClasses; ++LQ) {
                b->n_tiles[LP * kClasses + LQ] = (int)tl[LP][LQ].size();
                b->tiles[LP][LQ] = tl[LP][LQ].empty() ? nullptr : b->upload(tl[LP][LQ], s, "tiles");
            }
        // default tile plans (persistent queues) of the engines this context's builds use
        b->jplan = jplan_create(tl, frag_npp, pair_x, pair_y, c->device);
        ck(jplan_prepare(b->jplan, o.exact_engine == FEF_ENGINE_DF64 ? 2 : 0, s), "J-engine plan");
        if (o.precision == FEF_MIXED) ck(jplan_prepare(b->jplan, 1, s), "J-engine plan");
        c->prim_quartets = prim_q;
        const int ncount = 1 + kClasses * kClasses;
        b->qcount = b->alloc<unsigned long long>(ncount, "qcount");
        ck(cudaMemsetAsync(b->qcount, 0, sizeof(unsigned long long) * ncount, s), "qcount");
        ck(launch_count_quartets(d, o.schwarz, b->qcount, s), "count quartets");
        unsigned long long qc[1 + kClasses * kClasses] = {};
        ck(cudaMemcpyAsync(qc, b->qcount, sizeof(qc), cudaMemcpyDeviceToHost, s), "qcount");
        // per-build buffers
        b->D = b->alloc<double>(c->mat_total, "D");
        b->F = b->alloc<double>(c->mat_total, "F");
        b->Jenv = b->alloc<double>(c->mat_total, "Jenv");
        b->omega = b->alloc<double>(c->mat_total, "omega");
        ck(cudaMemsetAsync(b->D, 0, sizeof(double) * c->mat_total, s), "D");
        {   // nuclear trace fields: per (pair, direction) sum_L nh(L) npp_x[L] doubles
            std::vector<int64_t> off(2 * (size_t)c->n_pairs + 1, 0);
            for (int p = 0; p < c->n_pairs; ++p)
                for (int dir = 0; dir < 2; ++dir) {
                    const int x = dir == 0 ? pair_x[p] : pair_y[p];
                    int64_t w = 0;
                    for (int L = 0; L < kClasses; ++L) w += (int64_t)nh(L) * frag_npp[x * kClasses + L];
                    off[2 * p + dir + 1] = off[2 * p + dir] + w;
                }
            b->trf_off = b->upload(off, s, "trace fields");
            b->trf = b->alloc<double>(std::max<int64_t>(off.back(), 1), "trace fields");
            ck(launch_nuclear_trace_fields(d, b->trf_off, b->trf, s), "trace fields");
        }
        b->tr_xy = b->alloc<double>(c->n_pairs, "tr");
        b->tr_yx = b->alloc<double>(c->n_pairs, "tr");
        b->trV = b->alloc<double>(nf, "trV");
        b->trJ = b->alloc<double>(nf, "trJ");
        b->E_int = b->alloc<double>(nf, "E_int");
        b->E_scf = b->alloc<double>(nf, "E_scf");
        b->E_frag = b->alloc<double>(nf, "E_frag");
        b->E_tot = b->alloc<double>(1, "E_tot");
        ck(cudaMallocHost(&b->stage, 16 + 16 * (size_t)nf + 32), "pinned read-back");
        ck(cudaMallocHost(&b->scf_tol_host, 2 * sizeof(double)), "pinned thresholds");
        b->scf_tol = b->alloc<double>(2, "SCF thresholds");
        b->scf_tol_host[0] = o.micro_e_tol;
        b->scf_tol_host[1] = o.micro_comm_tol;
        ck(cudaMemcpyAsync(b->scf_tol, b->scf_tol_host, 2 * sizeof(double), cudaMemcpyHostToDevice, s), "thresholds");
        b->stamps = b->alloc<unsigned long long>(4, "timestamps");
        b->iters = b->alloc<int>(nf, "iters");
        b->gap = b->alloc<double>(nf, "gap");
        ck(cudaMemsetAsync(b->iters, 0, sizeof(int) * nf, s), "iters");
        ck(cudaMemsetAsync(b->gap, 0, sizeof(double) * nf, s), "gap");
        // DIIS history at 2 diis_size frag_moff[x] (sized per fragment); SCF workspace in global
        // memory only for fragments too large for shared memory
        b->diis_stride = 0;
        b->diis = b->alloc<double>(2 * (size_t)o.diis_size * c->mat_total, "diis");
        b->scf_ws = max_nao > kScfSmemMaxN ? b->alloc<double>(9 * c->mat_total, "SCF workspace") : nullptr;
        if (max_nao > kScfSmemMaxN) {
            std::vector<int> small, big;
            for (int x = 0; x < nf; ++x) (c->nao[x] > kScfSmemMaxN ? big : small).push_back(x);
            b->n_scf_small = (int)small.size();
            b->n_scf_big = (int)big.size();
            if (!small.empty()) b->scf_small = b->upload(small, s, "SCF lists");
            b->scf_big = b->upload(big, s, "SCF lists");
        }
        ck(cudaStreamSynchronize(s), "create");
        c->shell_quartets = (int64_t)qc[0];
        for (int i = 0; i < kClasses * kClasses; ++i) c->class_quartets[i] = (int64_t)qc[1 + i];
        check_device_flags(c, "create");
        *out = c;
        return FEF_OK;
    } catch (const Error& e) {
        g_create_error = e.msg;
        if (c) {
            delete c->buf;
            delete c;
        }
        return e.status;
    } catch (const std::exception& e) {
        g_create_error = e.what();
        if (c) {
            delete c->buf;
            delete c;
        }
        return FEF_ERR_ARG;
    }
}

extern "C" void fef_destroy(fef_ctx* c)
{
    if (!c) return;
    if (c->buf) {
        if (c->buf->ev0) cudaEventDestroy(c->buf->ev0);
        if (c->buf->ev1) cudaEventDestroy(c->buf->ev1);
        if (c->buf->ev2) cudaEventDestroy(c->buf->ev2);
        if (c->buf->ev3) cudaEventDestroy(c->buf->ev3);
        delete c->buf;
    }
    delete c;
}

extern "C" const char* fef_last_error(const fef_ctx* c)
{
    return c ? c->last_error.c_str() : g_create_error.c_str();
}

extern "C" fef_status fef_ao_layout(const fef_ctx* c, int32_t* n_ao_per_frag, int64_t* offsets)
{
    if (!c) return FEF_ERR_ARG;
    for (int x = 0; x < c->n_frag; ++x) {
        if (n_ao_per_frag) n_ao_per_frag[x] = c->nao[x];
        if (offsets) offsets[x] = c->moff[x];
    }
    if (offsets) offsets[c->n_frag] = c->moff[c->n_frag];
    return FEF_OK;
}

static void copy_packed(fef_ctx* c, double* dst, const double* src, int on_device, cudaMemcpyKind host_kind)
{
    size_t bytes = sizeof(double) * c->mat_total;
    ck(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : host_kind, c->stream), "copy");
    if (!on_device) ck(cudaStreamSynchronize(c->stream), "copy");
}

extern "C" fef_status fef_set_densities(fef_ctx* c, const double* D, int on_device)
{
    if (!c) return FEF_ERR_ARG;
    FEF_API_BEGIN
    require(D != nullptr, FEF_ERR_ARG, "fef_set_densities: NULL D");
    copy_packed(c, c->buf->D, D, on_device, cudaMemcpyHostToDevice);
    c->have_density = true;
    c->energies_valid = false;
    return FEF_OK;
    FEF_API_END(c)
}

extern "C" fef_status fef_get_densities(const fef_ctx* cc, double* D, int on_device)
{
    fef_ctx* c = const_cast<fef_ctx*>(cc);
    if (!c) return FEF_ERR_ARG;
    FEF_API_BEGIN
    require(D != nullptr, FEF_ERR_ARG, "fef_get_densities: NULL output");
    require(c->have_density, FEF_ERR_ARG, "fef_get_densities: no densities yet");
    copy_packed(c, D, c->buf->D, on_device, cudaMemcpyDeviceToHost);
    return FEF_OK;
    FEF_API_END(c)
}

extern "C" fef_status fef_build_fock(fef_ctx* c, const double* D, double* F_out, int on_device)
{
    if (!c) return FEF_ERR_ARG;
    FEF_API_BEGIN
    if (D) {
        copy_packed(c, c->buf->D, D, on_device, cudaMemcpyHostToDevice);
        c->have_density = true;
    }
    require(c->have_density, FEF_ERR_ARG, "fef_build_fock: no densities given or set");
    clear_flags(c);
    int kind = kBuildFP64;
    if (c->opt.precision == FEF_MIXED)
        kind = c->opt.mixed_build == FEF_MIXED_WHOLE ? kBuildFP32Ref : (c->buf->ref_exact ? kBuildFP32Inc : kBuildFP64);
    build_fock_internal(c, kind);
    if (F_out) copy_packed(c, F_out, c->buf->F, on_device, cudaMemcpyDeviceToHost);
    check_device_flags(c, "fef_build_fock");
    float ms = 0.f;
    ck(cudaEventElapsedTime(&ms, c->buf->ev0, c->buf->ev1), "event time");
    c->jengine_ms = ms;
    return FEF_OK;
    FEF_API_END(c)
}

static void read_energies(fef_ctx* c, std::vector<double>& Ex, double& Et)
{
    Ex.resize(c->n_frag);
    ck(cudaMemcpyAsync(Ex.data(), c->buf->E_frag, sizeof(double) * c->n_frag, cudaMemcpyDeviceToHost, c->stream),
       "energies");
    ck(cudaMemcpyAsync(&Et, c->buf->E_tot, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "energies");
    ck(cudaStreamSynchronize(c->stream), "energies");
}

static void ensure_learn_buffers(fef_ctx* c)
{
    require(c->learn_feat > 0, FEF_ERR_ARG,
            "learned warm start: fragments must all be of one kind (same atoms, s/p basis)");
    Buffers* b = c->buf;
    if (!b->Xd) {
        b->Xd = b->alloc<float>((size_t)c->n_frag * c->learn_feat, "learned X");
        b->Yd = b->alloc<float>((size_t)c->n_frag * c->learn_pack, "learned Y");
        b->D_iso = b->alloc<double>(c->mat_total, "D_iso");
        b->omega_mp = b->alloc<double>(c->mat_total, "multipole omega");
        b->desc_part = b->alloc<double>((size_t)std::max(c->n_nbr, 1) * c->learn_desc, "descriptor terms");
    }
}

// Features of the current densities into b->Xd, with no Fock build: the potential and field of the
// neighbours (nuclei and Hermite densities) at the atoms (columns [0, learn_desc)) and the multipole
// estimate of the environment operator (each neighbour's charge, dipole and second moments about its
// centroid, Taylor-expanded to second order about the fragment's centroid) in the Loewdin basis and
// molecule-fixed frame (columns [learn_desc, learn_feat)).
static void compute_features(fef_ctx* c)
{
    Buffers* b = c->buf;
    const Dev& d = c->dev;
    ck(launch_hermite_density(d, b->D, c->stream), "hermite density");
    ck(launch_descriptors(d, b->rot, c->learn_feat, c->learn_desc / 4, c->n_nbr, b->desc_part, b->Xd, c->stream),
       "descriptors");
    ck(launch_near_multipole_field(d, b->far_M, b->far_Mnuc, b->far_cen, b->D, b->far_mult, b->far_pot, b->omega_mp,
                                   c->mat_total, c->stream),
       "multipole environment operator");
    ck(launch_local_density(d, b->rot, b->Sih, b->omega_mp, c->learn_feat, c->learn_desc, b->Xd, c->stream),
       "environment operator");
}

// D <- D_iso + S^{-1/2} B f(features(D_iso)) B^T S^{-1/2}: the current densities are the isolated ones.
static void learned_start(fef_ctx* c)
{
    ensure_learn_buffers(c);
    Buffers* b = c->buf;
    require(mlp_n_in(c->warm_start) == c->learn_feat && mlp_n_out(c->warm_start) == c->learn_pack, FEF_ERR_ARG,
            "warm-start network dimensions do not match the fragments");
    ck(cudaMemcpyAsync(b->D_iso, b->D, sizeof(double) * c->mat_total, cudaMemcpyDeviceToDevice, c->stream), "D_iso");
    compute_features(c);
    ck(mlp_predict_device(c->warm_start, b->Xd, b->Yd, c->n_frag, c->stream), "warm-start network");
    ck(launch_apply_learned(c->dev, b->rot, b->Sih, b->D_iso, b->Yd, c->learn_pack, b->D, c->stream), "apply learned");
    c->energies_valid = false;
}

extern "C" fef_status fef_set_warm_start(fef_ctx* c, fef_mlp* m)
{
    if (!c) return FEF_ERR_ARG;
    FEF_API_BEGIN
    if (m) {
        require(c->learn_feat > 0, FEF_ERR_ARG,
                "learned warm start: fragments must all be of one kind (same atoms, s/p basis)");
        require(mlp_n_in(m) == c->learn_feat && mlp_n_out(m) == c->learn_pack, FEF_ERR_ARG,
                "warm-start network dimensions do not match the fragments");
    }
    c->warm_start = m;
    return FEF_OK;
    FEF_API_END(c)
}

extern "C" fef_status fef_learned_features(fef_ctx* c, const double* D, float* X, float* Y_local, int on_device,
                                           int32_t* n_feat, int32_t* n_pack)
{
    if (!c) return FEF_ERR_ARG;
    FEF_API_BEGIN
    if (n_feat) *n_feat = c->learn_feat;
    if (n_pack) *n_pack = c->learn_pack;
    if (!X && !Y_local) return FEF_OK;
    ensure_learn_buffers(c);
    Buffers* b = c->buf;
    if (D) {
        copy_packed(c, b->D, D, on_device, cudaMemcpyHostToDevice);
        c->have_density = true;
        c->energies_valid = false;
    }
    require(c->have_density, FEF_ERR_ARG, "fef_learned_features: no densities given or set");
    const size_t nx = (size_t)c->n_frag * c->learn_feat, ny = (size_t)c->n_frag * c->learn_pack;
    if (X) {
        compute_features(c);
        ck(cudaMemcpyAsync(X, b->Xd, sizeof(float) * nx, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                           c->stream), "X");
    }
    if (Y_local) {
        ck(launch_local_density(c->dev, b->rot, b->Sh, b->D, c->learn_pack, 0, b->Yd, c->stream), "local density");
        ck(cudaMemcpyAsync(Y_local, b->Yd, sizeof(float) * ny,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream), "Y");
    }
    ck(cudaStreamSynchronize(c->stream), "learned features");
    return FEF_OK;
    FEF_API_END(c)
}

extern "C" fef_status fef_noninteracting_scf(fef_ctx* c)
{
    if (!c) return FEF_ERR_ARG;
    FEF_API_BEGIN
    clear_flags(c);
    set_scf_thresholds(c, -1.0);
    run_scf(c, false, false);
    int flag = 0;
    ck(cudaMemcpyAsync(&flag, c->buf->err_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "flags");
    ck(cudaStreamSynchronize(c->stream), "isolated RHF");
    c->have_density = true;
    c->energies_valid = false;
    if (flag & kErrNumeric) throw Error{FEF_ERR_NUMERIC, "NaN/Inf in an isolated-fragment RHF"};
    if (flag & kErrNotConv) throw Error{FEF_ERR_NOT_CONVERGED, "isolated-fragment RHF did not converge"};
    return FEF_OK;
    FEF_API_END(c)
}

extern "C" fef_status fef_iterate(fef_ctx* c, int32_t* n_macro_out, double* final_dE_out)
{
    if (!c) return FEF_ERR_ARG;
    FEF_API_BEGIN
    const fef_options& o = c->opt;
    clear_flags(c);
    if (o.start == FEF_START_GIVEN) {
        require(c->have_density, FEF_ERR_ARG, "fef_iterate: start=GIVEN but no densities were set");
    } else if (o.start == FEF_START_SUPERPOSITION) {
        set_scf_thresholds(c, -1.0);
        run_scf(c, false, false);  // isolated-fragment RHF from the core guess
        int flag = 0;
        ck(cudaMemcpyAsync(&flag, c->buf->err_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "flags");
        ck(cudaStreamSynchronize(c->stream), "isolated RHF");
        if (flag & kErrNotConv) throw Error{FEF_ERR_NOT_CONVERGED, "isolated-fragment RHF did not converge"};
        c->have_density = true;
    } else {
        // learned: isolated-fragment RHF, then D = D_iso + the network's predicted change from the
        // environment potential and field at each atom (molecule-fixed frames)
        require(c->warm_start != nullptr, FEF_ERR_ARG, "fef_iterate: start=LEARNED needs fef_set_warm_start");
        set_scf_thresholds(c, -1.0);
        run_scf(c, false, false);
        int flag = 0;
        ck(cudaMemcpyAsync(&flag, c->buf->err_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "flags");
        ck(cudaStreamSynchronize(c->stream), "isolated RHF");
        if (flag & kErrNotConv) throw Error{FEF_ERR_NOT_CONVERGED, "isolated-fragment RHF did not converge"};
        learned_start(c);
        c->have_density = true;
    }
    double it_max = 0, it_sum = 0, scf_ms = 0;
    if (o.start != FEF_START_GIVEN) scf_counts(c, it_max, it_sum, scf_ms);
    check_device_flags(c, "fef_iterate start");
    // MIXED: the first field is an FP32-core reference and the coarse phase follows, from any start.
    // (An exact reference built at a learned start would sit at a density that is not idempotent
    // and still ~1e-3 from the fixed point; the fine increments relative to it then carry enough
    // FP32 error to stall near e_tol and force further exact builds.)
    const bool mixed = (o.precision == FEF_MIXED);
    build_fock_internal(c, mixed ? kBuildFP32Ref : kBuildFP64);
    std::vector<double> Ex_old, Ex;
    double Et_old = 0, Et = 0, dE = 0;
    read_energies(c, Ex_old, Et_old);
    c->history.clear();
    float jms = 0.f;
    {
        float ms0 = 0.f;
        ck(cudaEventElapsedTime(&ms0, c->buf->ev0, c->buf->ev1), "event time");
        double rec[kHistoryFields] = {0, Et_old, 0, 0, it_max, it_sum, ms0, scf_ms, c->last_build_fp32 ? 1.0 : 0.0};
        c->history.insert(c->history.end(), rec, rec + kHistoryFields);
        jms = ms0;
    }
    int k = 0;
    bool conv = false;
    // MIXED: a coarse phase of FP32-core increments relative to the FP32 reference field, until
    // the energy changes fall below mixed_switch or stop decreasing; then one FP64 build becomes the
    // exact reference and the fine phase continues with FP32 increments relative to it, whose error
    // (it grows with |D - D_ref|) is now far below e_tol.  Convergence is declared only between two
    // consecutive accurate energies (FP64, or FP32 increments on an exact reference); a stalled fine
    // phase refreshes the reference again.
    bool fine = !mixed;
    bool next_fp32 = mixed;
    bool prev_acc = !c->last_build_fp32;
    double dE_prev = 1e300;
    // fragment-SCF thresholds follow the previous macro-iteration's energy change (the first one,
    // from the isolated or given densities, assumes a 1e-3 Eh polarisation step)
    double prog_last = 1e-3;
    for (k = 1; k <= o.max_macro; ++k) {
        const int kind = resolve_kind(c, next_fp32 ? kBuildFP32Inc : kBuildFP64);
        set_scf_thresholds(c, prog_last);
        macro_step(c, kind);
        build_fock_host(c, kind);
        const bool this_fp64 = !c->last_build_fp32;
        const bool this_acc = this_fp64 || (fine && c->buf->ref_exact);
        Et = *stage_Et(c);
        Ex.assign(stage_Ex(c), stage_Ex(c) + c->n_frag);
        it_max = 0;
        it_sum = 0;
        for (int x = 0; x < c->n_frag; ++x) {
            it_max = std::max<double>(it_max, std::abs(stage_iters(c)[x]));
            it_sum += std::abs(stage_iters(c)[x]);
        }
        float ms = 0.f, sms = 0.f;
        if (o.use_graph) {  // device timestamps of the graph's phase marks
            const unsigned long long* t = stage_stamps(c);
            ms = (float)((t[1] - t[0]) * 1e-6);
            sms = (float)((t[3] - t[2]) * 1e-6);
        } else {
            ck(cudaEventElapsedTime(&ms, c->buf->ev0, c->buf->ev1), "event time");
            ck(cudaEventElapsedTime(&sms, c->buf->ev2, c->buf->ev3), "event time");
        }
        scf_ms = sms;
        jms += ms;
        const int flag = *stage_flag(c);
        if (flag & kErrNumeric) throw Error{FEF_ERR_NUMERIC, "NaN/Inf during FEF iteration"};
        if (flag & kErrNotConv)
            throw Error{FEF_ERR_NOT_CONVERGED, "fragment RHF in the field did not converge at macro-iteration " +
                                                   std::to_string(k)};
        dE = std::fabs(Et - Et_old);
        double dEx = 0;
        for (int x = 0; x < c->n_frag; ++x) dEx = std::max(dEx, std::fabs(Ex[x] - Ex_old[x]));
        {
            double rec[kHistoryFields] = {(double)k, Et, dE, dEx, it_max, it_sum, (double)ms, scf_ms,
                                          this_fp64 ? 0.0 : 1.0};
            c->history.insert(c->history.end(), rec, rec + kHistoryFields);
        }
        Ex_old = Ex;
        Et_old = Et;
        if (this_acc && prev_acc && dE < o.e_tol && dEx < o.e_tol) {
            conv = true;
            break;
        }
        // progress measure: the larger of |dE_tot| and max_x |dE_x| (|dE_tot| alone can drop by
        // cancellation between fragments and then rise again without any stall)
        const double prog = std::max(dE, dEx);
        prog_last = prog;
        if (mixed) {
            if (!fine) {
                if (prog < o.mixed_switch || prog > dE_prev) {
                    fine = true;        // refresh the FP64 reference next
                    next_fp32 = false;
                }
            } else if (this_fp64) {
                next_fp32 = true;       // fine increments relative to the fresh reference
            } else if (prog > dE_prev) {
                next_fp32 = false;      // stalled: refresh again
            }
        }
        prev_acc = this_acc;
        dE_prev = prog;
    }
    c->jengine_ms = jms;
    if (n_macro_out) *n_macro_out = conv ? k : o.max_macro;
    if (final_dE_out) *final_dE_out = dE;
    if (!conv) throw Error{FEF_ERR_NOT_CONVERGED, "FEF did not converge within max_macro"};
    return FEF_OK;
    FEF_API_END(c)
}

extern "C" fef_status fef_energies(fef_ctx* c, double* E_frag, double* E_total, double* E_int)
{
    if (!c) return FEF_ERR_ARG;
    FEF_API_BEGIN
    require(c->have_density, FEF_ERR_ARG, "fef_energies: no densities");
    if (!c->energies_valid) {
        clear_flags(c);
        build_fock_internal(c);
    }
    if (E_frag)
        ck(cudaMemcpyAsync(E_frag, c->buf->E_frag, sizeof(double) * c->n_frag, cudaMemcpyDeviceToHost, c->stream), "E");
    if (E_total) ck(cudaMemcpyAsync(E_total, c->buf->E_tot, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "E");
    if (E_int)
        ck(cudaMemcpyAsync(E_int, c->buf->E_int, sizeof(double) * c->n_frag, cudaMemcpyDeviceToHost, c->stream), "E");
    ck(cudaStreamSynchronize(c->stream), "energies");
    check_device_flags(c, "fef_energies");
    return FEF_OK;
    FEF_API_END(c)
}

extern "C" fef_status fef_stats(const fef_ctx* c, int64_t* sq, int64_t* pq, int64_t* np, double* jms,
                                int64_t* launches, int64_t* class_quartets)
{
    if (launches) *launches = launches_so_far();
    if (!c) return launches ? FEF_OK : FEF_ERR_ARG;
    if (class_quartets)
        for (int i = 0; i < kClasses * kClasses; ++i) class_quartets[i] = c->class_quartets[i];
    if (sq) *sq = c->shell_quartets;
    if (pq) *pq = c->prim_quartets;
    if (np) *np = c->n_pairs;
    if (jms) *jms = c->jengine_ms;
    return FEF_OK;
}

extern "C" fef_status fef_measure_fma_peak(double* fp64, double* fp32, double* mhz)
{
    cudaError_t e = measure_fma_peak(fp64, fp32, mhz);
    if (e != cudaSuccess) {
        g_create_error = std::string("fef_measure_fma_peak: ") + cudaGetErrorString(e);
        return FEF_ERR_CUDA;
    }
    return FEF_OK;
}

extern "C" fef_status fef_history(const fef_ctx* c, int32_t max_records, double* records, int32_t* n_records)
{
    if (!c) return FEF_ERR_ARG;
    int n = (int)(c->history.size() / kHistoryFields);
    if (n_records) *n_records = n;
    if (records && max_records > 0) {
        int m = std::min(n, (int)max_records);
        std::memcpy(records, c->history.data(), sizeof(double) * kHistoryFields * m);
    }
    return FEF_OK;
}

extern "C" fef_status fef_get_tile_plan(const fef_ctx* c, int32_t engine, fef_tile_plan* out)
{
    if (!c || !out || engine < 0 || engine > 2) return FEF_ERR_ARG;
    jplan_get(c->buf->jplan, engine, out);
    return FEF_OK;
}

extern "C" fef_status fef_set_tile_plan(fef_ctx* c, int32_t engine, const fef_tile_plan* plan)
{
    if (!c) return FEF_ERR_ARG;
    FEF_API_BEGIN
    require(plan != nullptr && engine >= 0 && engine <= 2 && plan->persistent >= 0 && plan->persistent <= 2,
            FEF_ERR_ARG, "fef_set_tile_plan: bad engine or plan");
    for (int i = 0; i < 25; ++i)
        require(plan->ket_chunk[i] >= 0 && plan->ket_chunk[i] < (1 << 26), FEF_ERR_ARG,
                "fef_set_tile_plan: ket_chunk out of range");
    ck(cudaStreamSynchronize(c->stream), "tile plan");
    ck(jplan_set(c->buf->jplan, engine, plan, c->stream), "tile plan");
    for (auto& g : c->buf->macro_graph)  // graphs captured with the old queues are stale
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    return FEF_OK;
    FEF_API_END(c)
}

extern "C" fef_status fef_autotune(fef_ctx* c, int32_t engine, int32_t reps, double budget_ms, fef_tile_plan* out)
{
    if (!c) return FEF_ERR_ARG;
    FEF_API_BEGIN
    require(engine >= 0 && engine <= 2 && reps >= 1 && reps <= 100 && budget_ms > 0.0, FEF_ERR_ARG,
            "fef_autotune: bad engine, reps or budget");
    Buffers* b = c->buf;
    ck(cudaStreamSynchronize(c->stream), "autotune");
    // the engine's inputs from the current densities (the same preparation as a build of that
    // engine, relative to the stored reference for FP32), so that the timed passes see the
    // context's own pair data and weights; the reference itself is left unchanged
    const Dev& d = c->dev;
    ck(launch_hermite_density(d, b->D, c->stream), "autotune: hermite density");
    if (engine == 1) {
        ck(launch_fp32_records(d, b->Dh_ref, b->rec_resid, c->stream), "autotune: fp32 records");
    } else if (engine == 2) {
        ck(launch_df_density(d, c->stream), "autotune: df64 density");
    }
    const int2* tiles[kClasses][kClasses];
    for (int i = 0; i < kClasses; ++i)
        for (int j = 0; j < kClasses; ++j) tiles[i][j] = b->tiles[i][j];
    ck(jplan_autotune(b->jplan, c->dev, engine, tiles, b->n_tiles, c->opt.schwarz, reps, budget_ms, c->stream, out),
       "autotune");
    // the queues changed: graphs captured with the old ones are stale
    for (auto& g : b->macro_graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    return FEF_OK;
    FEF_API_END(c)
}

extern "C" fef_status fef_fragment_status(const fef_ctx* cc, int32_t* micro_iters, double* homo_lumo_gap,
                                          double* E_scf)
{
    if (!cc) return FEF_ERR_ARG;
    fef_ctx* c = const_cast<fef_ctx*>(cc);
    FEF_API_BEGIN
    Buffers* b = c->buf;
    const int nf = c->n_frag;
    if (micro_iters)
        ck(cudaMemcpyAsync(micro_iters, b->iters, sizeof(int) * nf, cudaMemcpyDeviceToHost, c->stream), "status");
    if (homo_lumo_gap)
        ck(cudaMemcpyAsync(homo_lumo_gap, b->gap, sizeof(double) * nf, cudaMemcpyDeviceToHost, c->stream), "status");
    if (E_scf) ck(cudaMemcpyAsync(E_scf, b->E_scf, sizeof(double) * nf, cudaMemcpyDeviceToHost, c->stream), "status");
    ck(cudaStreamSynchronize(c->stream), "status");
    return FEF_OK;
    FEF_API_END(c)
}

extern "C" fef_status fef_energy_m2(fef_ctx* c, double* E_m2, double* E_m2_total)
{
    if (!c) return FEF_ERR_ARG;
    FEF_API_BEGIN
    require(c->have_density, FEF_ERR_ARG, "fef_energy_m2: no densities");
    Buffers* b = c->buf;
    const Dev& d = c->dev;
    cudaStream_t s = c->stream;
    const int nf = c->n_frag;
    if (!c->energies_valid) build_fock_internal(c, kBuildFP64);  // F of the current densities
    // intra-fragment (mu nu|lambda sigma), pair-packed, recomputed into a temporary
    std::vector<int4> tasks;
    std::vector<int> cls_off;
    intra_eri_tasks(nf, c->h_frag_sp0, c->h_sp_a, c->h_sp_b, c->h_sh_l, tasks, cls_off);
    std::vector<int64_t> off(nf + 1, 0);
    for (int x = 0; x < nf; ++x) off[x + 1] = off[x] + energy_m2_workspace(c->nao[x], c->nocc[x], c->nmo[x]);
    double* U = b->alloc<double>(std::max<int64_t>(c->coff_total, 1), "E_M2 integrals");
    int4* tasks_d = b->upload(tasks, s, "E_M2 tasks");
    int64_t* off_d = b->upload(off, s, "E_M2 offsets");
    double* ws = b->alloc<double>(std::max<int64_t>(off[nf], 1), "E_M2 workspace");
    double* E_d = b->alloc<double>(nf, "E_M2");
    std::vector<double> E(nf, 0.0);
    cudaError_t e = launch_intra_eri(d, tasks_d, cls_off, U, s);
    if (e == cudaSuccess) e = launch_energy_m2(d, b->F, b->X, b->nmo, U, off_d, ws, E_d, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(E.data(), E_d, sizeof(double) * nf, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    b->release(U);
    b->release(tasks_d);
    b->release(off_d);
    b->release(ws);
    b->release(E_d);
    ck(e, "fef_energy_m2");
    double tot = 0.0;
    for (double v : E) tot += v;
    if (E_m2) std::copy(E.begin(), E.end(), E_m2);
    if (E_m2_total) *E_m2_total = tot;
    return FEF_OK;
    FEF_API_END(c)
}

extern "C" fef_status fef_energy_d2(fef_ctx* c, double* E_d2_frag, double* E_d2_total)
{
    if (!c) return FEF_ERR_ARG;
    FEF_API_BEGIN
    require(c->have_density, FEF_ERR_ARG, "fef_energy_d2: no densities");
    Buffers* b = c->buf;
    const Dev& d = c->dev;
    cudaStream_t s = c->stream;
    const int nf = c->n_frag;
    if (!c->energies_valid) build_fock_internal(c, kBuildFP64);  // F of the current densities
    int nao_total = 0;
    for (int x = 0; x < nf; ++x) nao_total += c->nao[x];
    double* C = b->alloc<double>(std::max<int64_t>(c->mat_total, 1), "E_D2 orbitals");
    double* eps = b->alloc<double>(std::max(nao_total, 1), "E_D2 orbital energies");
    double* jws = b->alloc<double>(std::max<int64_t>(2 * c->mat_total, 1), "E_D2 Jacobi workspace");
    std::vector<double> E_pair(c->n_pairs, 0.0);
    cudaError_t e = launch_canonical_orbitals(d, b->F, b->X, b->nmo, jws, C, eps, s);
    // s/p fragments: transition Hermite densities and the many-density J-engine (ed2.cu)
    bool sp_only = true;
    for (int x = 0; x < nf; ++x)
        for (int L = 3; L < kClasses; ++L) sp_only = sp_only && c->h_frag_npp[x * kClasses + L] == 0;
    if (sp_only && e == cudaSuccess) {
        std::vector<int> n_ov(nf), hoff(nf * kClasses), n_herm(nf);
        std::vector<int64_t> uoff(nf + 1, 0);
        int max_ov = 1;
        for (int x = 0; x < nf; ++x) {
            n_ov[x] = c->nocc[x] * (c->nmo[x] - c->nocc[x]);
            max_ov = std::max(max_ov, n_ov[x]);
            int hsum = 0;
            for (int L = 0; L < kClasses; ++L) {
                hoff[x * kClasses + L] = hsum;
                hsum += c->h_frag_npp[x * kClasses + L] * nh(L);
            }
            n_herm[x] = hsum;
            uoff[x + 1] = uoff[x] + (int64_t)hsum * n_ov[x];
        }
        int* n_ov_d = b->upload(n_ov, s, "E_D2 sizes");
        int* hoff_d = b->upload(hoff, s, "E_D2 sizes");
        int* nherm_d = b->upload(n_herm, s, "E_D2 sizes");
        int64_t* uoff_d = b->upload(uoff, s, "E_D2 sizes");
        double* U = b->alloc<double>(std::max<int64_t>(uoff[nf], 1), "E_D2 transition densities");
        e = launch_ed2_transition(d, C, b->nmo, uoff_d, hoff_d, n_ov_d, max_ov, U, s);
        float2* Udf = b->alloc<float2>(std::max<int64_t>(uoff[nf], 1), "E_D2 transition densities (float-float)");
        if (e == cudaSuccess) e = launch_ed2_split(U, Udf, uoff[nf], s);
        const int64_t kMaxG = 1ll << 27;
        std::vector<int> chunk;
        std::vector<int64_t> goff(1, 0);
        std::vector<int4> items[3];
        int max_entries = 1;  // largest n_ov(x) n_ov(y) of the chunk's pairs
        auto run = [&]() {
            if (chunk.empty() || e != cudaSuccess) return;
            const int nq = (int)chunk.size();
            int* pair_d = b->upload(chunk, s, "E_D2 pairs");
            int64_t* goff_d = b->upload(goff, s, "E_D2 offsets");
            double* G = b->alloc<double>(std::max<int64_t>(goff.back(), 1), "E_D2 fields");
            int4* items_d[3] = {};
            int n_items[3];
            for (int L = 0; L < 3; ++L) {
                n_items[L] = (int)items[L].size();
                if (n_items[L]) items_d[L] = b->upload(items[L], s, "E_D2 items");
            }
            const int ns = ed2_energy_slices(max_entries);
            double* Ed = b->alloc<double>((int64_t)nq * ns, "E_D2");
            std::vector<double> Eh((size_t)nq * ns);
            e = cudaMemsetAsync(G, 0, sizeof(double) * std::max<int64_t>(goff.back(), 1), s);
            const int4* cit[3] = {items_d[0], items_d[1], items_d[2]};
            if (e == cudaSuccess)
                e = launch_ed2_pairs(d, U, Udf, uoff_d, hoff_d, n_ov_d, pair_d, goff_d, G, c->opt.schwarz, cit, n_items,
                                     s);
            if (e == cudaSuccess)
                e = launch_ed2_energy(d, nq, max_entries, U, uoff_d, hoff_d, n_ov_d, pair_d, goff_d, G, C, eps, b->nmo,
                                      nherm_d, Ed, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(Eh.data(), Ed, sizeof(double) * Eh.size(), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            for (int q = 0; q < nq; ++q) {
                double sum = 0.0;
                for (int k = 0; k < ns; ++k) sum += Eh[(size_t)q * ns + k];
                E_pair[chunk[q]] = sum;
            }
            for (void* p : {(void*)pair_d, (void*)goff_d, (void*)G, (void*)Ed, (void*)items_d[0], (void*)items_d[1],
                            (void*)items_d[2]})
                if (p) b->release(p);
            chunk.clear();
            goff.assign(1, 0);
            for (auto& v : items) v.clear();
            max_entries = 1;
        };
        for (int p = 0; p < c->n_pairs && e == cudaSuccess; ++p) {
            const int x = c->h_pair_x[p], y = c->h_pair_y[p];
            const int64_t gx = (int64_t)n_herm[x] * n_ov[y], gy = (int64_t)n_herm[y] * n_ov[x];
            if (!chunk.empty() && goff.back() + gx + gy > kMaxG) run();
            const int q = (int)chunk.size();
            chunk.push_back(p);
            max_entries = std::max(max_entries, n_ov[x] * n_ov[y]);
            goff.push_back(goff.back() + gx);   // side 0: rows of x, columns jb of y
            goff.push_back(goff.back() + gy);   // side 1: rows of y, columns ia of x
            for (int side = 0; side < 2; ++side) {
                const int bx = side ? y : x, ky = side ? x : y;
                for (int LB = 0; LB < 3; ++LB) {
                    bool any_ket = false;  // ket classes >= LB (side 0) or > LB (side 1)
                    for (int LK = side ? LB + 1 : LB; LK < 3; ++LK) any_ket |= c->h_frag_npp[ky * kClasses + LK] > 0;
                    const int nb = c->h_frag_npp[bx * kClasses + LB];
                    if (!any_ket || nb == 0 || n_ov[ky] == 0) continue;
                    const int jc = ed2_cols_per_item(LB);
                    for (int o = 0; o < nb; o += 32)
                        for (int j0 = 0; j0 < n_ov[ky]; j0 += jc)
                            items[LB].push_back(make_int4(2 * q + side, c->h_frag_pp0[bx * kClasses + LB] + o, j0, 0));
                }
            }
        }
        run();
        b->release(U);
        b->release(Udf);
        for (void* p : {(void*)n_ov_d, (void*)hoff_d, (void*)nherm_d, (void*)uoff_d}) b->release(p);
    }
    // pairs in chunks that bound the integral blocks, workspaces and task lists
    const int64_t kMaxChunkDoubles = 1ll << 27, kMaxChunkTasks = 1ll << 24;
    std::vector<int> chunk;
    std::vector<int64_t> woff(1, 0), toff(1, 0);
    std::vector<int4> tasks;
    auto flush = [&]() {
        if (chunk.empty() || e != cudaSuccess) return;
        const int nq = (int)chunk.size();
        int* pair_d = b->upload(chunk, s, "E_D2 pairs");
        int64_t* woff_d = b->upload(woff, s, "E_D2 offsets");
        int64_t* toff_d = b->upload(toff, s, "E_D2 offsets");
        int4* tasks_d = b->upload(tasks, s, "E_D2 tasks");
        double* W = b->alloc<double>(std::max<int64_t>(woff.back(), 1), "E_D2 pair integrals");
        double* T = b->alloc<double>(std::max<int64_t>(toff.back(), 1), "E_D2 workspace");
        double* Ed = b->alloc<double>(nq, "E_D2");
        std::vector<double> Eh(nq);
        e = launch_pair_eri(d, tasks_d, (int)tasks.size(), pair_d, woff_d, W, s);
        if (e == cudaSuccess) e = launch_energy_d2(d, nq, pair_d, woff_d, W, C, eps, b->nmo, toff_d, T, Ed, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(Eh.data(), Ed, sizeof(double) * nq, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        for (int q = 0; q < nq; ++q) E_pair[chunk[q]] = Eh[q];
        for (void* p : {(void*)pair_d, (void*)woff_d, (void*)toff_d, (void*)tasks_d, (void*)W, (void*)T, (void*)Ed})
            b->release(p);
        chunk.clear();
        woff.assign(1, 0);
        toff.assign(1, 0);
        tasks.clear();
    };
    for (int p = 0; p < c->n_pairs && e == cudaSuccess && !sp_only; ++p) {
        const int x = c->h_pair_x[p], y = c->h_pair_y[p];
        const int nx = c->nao[x], ny = c->nao[y];
        const int64_t wsz = ((int64_t)nx * (nx + 1) / 2) * ((int64_t)ny * (ny + 1) / 2);
        const int64_t tsz = energy_d2_workspace(nx, c->nocc[x], c->nmo[x], ny, c->nocc[y], c->nmo[y]);
        int64_t ntask = 0;
        for (int s1 = c->h_frag_sp0[x]; s1 < c->h_frag_sp0[x + 1]; ++s1)
            ntask += (int64_t)ncart(c->h_sh_l[c->h_sp_a[s1]]) * ncart(c->h_sh_l[c->h_sp_b[s1]]) *
                     (c->h_frag_sp0[y + 1] - c->h_frag_sp0[y]);
        if (!chunk.empty() && (woff.back() + wsz + toff.back() + tsz > kMaxChunkDoubles ||
                               (int64_t)tasks.size() + ntask > kMaxChunkTasks))
            flush();
        const int q = (int)chunk.size();
        chunk.push_back(p);
        woff.push_back(woff.back() + wsz);
        toff.push_back(toff.back() + tsz);
        for (int s1 = c->h_frag_sp0[x]; s1 < c->h_frag_sp0[x + 1]; ++s1) {
            const int nk = ncart(c->h_sh_l[c->h_sp_a[s1]]) * ncart(c->h_sh_l[c->h_sp_b[s1]]);
            for (int s2 = c->h_frag_sp0[y]; s2 < c->h_frag_sp0[y + 1]; ++s2)
                for (int k = 0; k < nk; ++k) tasks.push_back(make_int4(q, s1, s2, k));
        }
    }
    flush();
    b->release(C);
    b->release(eps);
    b->release(jws);
    ck(e, "fef_energy_d2");
    double tot = 0.0;
    std::vector<double> Ef(nf, 0.0);
    for (int p = 0; p < c->n_pairs; ++p) {
        tot += E_pair[p];
        Ef[c->h_pair_x[p]] += 0.5 * E_pair[p];
        Ef[c->h_pair_y[p]] += 0.5 * E_pair[p];
    }
    if (E_d2_frag) std::copy(Ef.begin(), Ef.end(), E_d2_frag);
    if (E_d2_total) *E_d2_total = tot;
    return FEF_OK;
    FEF_API_END(c)
}
