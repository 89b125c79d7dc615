// Tile plans of the inter-fragment J-engine: how the work of one Fock build is cut into warp-sized
// items and launched.  The arithmetic is the same in every plan (paper, "Fragment Mean Field",
// Eq. wc / Eq. dp2e: J[D^y] over the surviving shell quartets); only the decomposition and the
// order of the floating-point additions change.
//
// A work item is one warp-tile of 32 bra primitive pairs of class L_P in one fragment of a pair
// against a chunk of the partner's primitive pairs of class L_Q (L_Q <= L_P).  Per engine (FP64
// core, FP32 core, float-float) a plan holds
//   * the strategy: persistent kernels over cost-sorted queues, or one launch per class pair;
//   * per class pair, the ket chunk (ket pairs per item; 0 = the whole class range).
// Persistent strategy: the items of all fragment pairs and classes are sorted by decreasing
// estimated cost (ket pairs x the algorithmic flops of one primitive quartet of the class) and split
// into register tiers — register-resident Hermite integrals (L_P + L_Q <= 4) and shared-memory ones
// (L_P + L_Q >= 5), plus the float-float s/p tier of that engine — each one persistent launch whose
// grid is the kernel's resident capacity; the tiers run on forked streams (graph branches when
// captured) so that a tier's tail overlaps the others.
// The autotuner times candidate plans on the context's own workload (CUDA events) and keeps the
// fastest: strategy, then the ket chunk of each class pair in decreasing order of class cost.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "internal.hpp"

namespace fef {

namespace {

constexpr int kNumCls = kClasses * kClasses;
constexpr int kChunkCandidates[] = {0, 1024, 256, 64};

// Algorithmic flops of one primitive quartet: setup + Boys + R recursion + both contractions
// (the cost key of the queue order).
double quartet_flops(int LP, int LQ)
{
    double f = 40.0;
    for (int k = 0; k <= LP + LQ; ++k) f += 3.0 * nh(k);
    return f + 2.0 * nh(LP) * nh(LQ);
}

bool is_big(int LP, int LQ) { return LP + LQ >= 5; }

struct Queue {
    int4* items = nullptr;
    int* next = nullptr;
    size_t cap = 0;
    int n = 0;
    int grid = 0;
    int slice = 0;
    bool spd = false;
};

constexpr int kSmallChunk = 64;  // ket pairs per work item on small workloads (jplan_create)

struct Plan {
    bool built = false;
    int persistent = 1;
    int chunk[kNumCls] = {};
    double tuned_ms = 0.0;
    Queue q[3];  // 0: register tier (FP64/FP32 core), 1: float-float s/p tier, 2: shared-memory tier
};

}  // namespace

struct JPlanSet {
    std::vector<int2> tiles[kNumCls];  // legacy tile list per class pair: (2 pair + swap, first bra pair)
    std::vector<int> nk[kNumCls];      // ket pairs of the partner per tile
    int n_sm = 0;
    Plan plan[3];
    cudaStream_t side[2] = {};
    cudaEvent_t fork = nullptr, join[2] = {};
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    ~JPlanSet()
    {
        for (auto& p : plan)
            for (auto& q : p.q) {
                if (q.items) cudaFree(q.items);
                if (q.next) cudaFree(q.next);
            }
        for (auto& st : side)
            if (st) cudaStreamDestroy(st);
        if (fork) cudaEventDestroy(fork);
        for (auto& e : join)
            if (e) cudaEventDestroy(e);
        if (t0) cudaEventDestroy(t0);
        if (t1) cudaEventDestroy(t1);
    }
};

namespace {

// Tier of class pair cls for engine mode: 0 register, 1 float-float, 2 shared memory.
int tier_of(int mode, int LP, int LQ)
{
    if (is_big(LP, LQ)) return 2;
    if (mode == 2 && LP <= 2) return 1;
    return 0;
}

// Host item lists of a plan (pairs with pair % stride == 0 only), sorted by decreasing cost.
void make_items(const JPlanSet& P, int mode, const int* chunk, int stride, std::vector<int4> out[3], bool spd[3],
                int slice[3])
{
    struct Keyed {
        double cost;
        int4 it;
    };
    std::vector<Keyed> tmp[3];
    for (int t = 0; t < 3; ++t) {
        spd[t] = false;
        slice[t] = 0;
    }
    for (int cls = 0; cls < kNumCls; ++cls) {
        const int LP = cls / kClasses, LQ = cls % kClasses;
        const auto& tl = P.tiles[cls];
        if (tl.empty()) continue;
        const int t = tier_of(mode, LP, LQ);
        const double f = quartet_flops(LP, LQ);
        if (t == 0 && LP >= 3) spd[t] = true;
        if (t == 2) slice[t] = std::max(slice[t], jengine_big_slice(LP, LQ));
        for (size_t i = 0; i < tl.size(); ++i) {
            if (stride > 1 && ((tl[i].x >> 1) % stride) != 0) continue;
            const int nk = P.nk[cls][i];
            const int c = chunk[cls] > 0 ? chunk[cls] : nk;
            for (int kb = 0; kb < nk; kb += c) {
                const int ke = std::min(nk, kb + c);
                tmp[t].push_back({f * (ke - kb), make_int4(tl[i].x, tl[i].y, kb, (ke << kItemClassBits) | cls)});
            }
        }
    }
    for (int t = 0; t < 3; ++t) {
        std::stable_sort(tmp[t].begin(), tmp[t].end(), [](const Keyed& a, const Keyed& b) { return a.cost > b.cost; });
        out[t].resize(tmp[t].size());
        for (size_t i = 0; i < tmp[t].size(); ++i) out[t][i] = tmp[t][i].it;
    }
}

cudaError_t tier_grid(int mode, int tier, bool spd, int slice, int* blocks_per_sm)
{
    if (tier == 0) return jengine_persistent_grid(mode == 1 ? 1 : 0, spd, blocks_per_sm);
    if (tier == 1) return jengine_df_persistent_grid(blocks_per_sm);
    return jengine_big_persistent_grid(mode == 1 ? 1 : 0, slice, blocks_per_sm);
}

// Build (or rebuild) the device queues of plan `mode` for its chunks.  Synchronous upload.
cudaError_t upload_plan(JPlanSet& P, int mode, int stride, cudaStream_t s)
{
    Plan& pl = P.plan[mode];
    std::vector<int4> items[3];
    bool spd[3];
    int slice[3];
    make_items(P, mode, pl.chunk, stride, items, spd, slice);
    for (int t = 0; t < 3; ++t) {
        Queue& q = pl.q[t];
        q.n = (int)items[t].size();
        q.spd = spd[t];
        q.slice = slice[t];
        if (q.n == 0) continue;
        if (items[t].size() > q.cap) {
            if (q.items) cudaFree(q.items);
            q.items = nullptr;
            cudaError_t e = cudaMalloc(&q.items, sizeof(int4) * items[t].size());
            if (e != cudaSuccess) return e;
            q.cap = items[t].size();
        }
        if (!q.next) {
            cudaError_t e = cudaMalloc(&q.next, sizeof(int));
            if (e != cudaSuccess) return e;
        }
        cudaError_t e = cudaMemcpyAsync(q.items, items[t].data(), sizeof(int4) * items[t].size(),
                                        cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return e;
        int bps = 0;
        e = tier_grid(mode, t, q.spd, q.slice, &bps);
        if (e != cudaSuccess) return e;
        q.grid = std::max(1, bps) * P.n_sm;
    }
    pl.built = true;
    return cudaStreamSynchronize(s);
}

JQueue as_jqueue(const Queue& q)
{
    JQueue j;
    j.items = q.items;
    j.n = q.n;
    j.next = q.next;
    j.grid = q.grid;
    j.smem_slice = q.slice;
    return j;
}

cudaError_t launch_tier(const Dev& d, int mode, int tier, const Queue& q, float tau, cudaStream_t s)
{
    const JQueue j = as_jqueue(q);
    if (tier == 0) return launch_jengine_persistent(d, mode == 1 ? 1 : 0, q.spd, j, tau, s);
    if (tier == 1) return launch_jengine_df_persistent(d, j, tau, s);
    return launch_jengine_big_persistent(d, mode == 1 ? 1 : 0, j, tau, s);
}

cudaError_t launch_persistent(JPlanSet& P, const Dev& d, int mode, float tau, cudaStream_t s)
{
    Plan& pl = P.plan[mode];
    // launch order: shared-memory tier (longest items) first, then the register and float-float tiers
    const int order[3] = {2, 0, 1};
    int active[3], na = 0;
    for (int t : order)
        if (pl.q[t].n > 0) active[na++] = t;
    if (na == 0) return cudaSuccess;
    if (na == 1) return launch_tier(d, mode, active[0], pl.q[active[0]], tau, s);
    cudaError_t e = cudaEventRecord(P.fork, s);
    if (e != cudaSuccess) return e;
    for (int i = 1; i < na; ++i) {
        e = cudaStreamWaitEvent(P.side[i - 1], P.fork, 0);
        if (e != cudaSuccess) return e;
    }
    for (int i = 0; i < na; ++i) {
        e = launch_tier(d, mode, active[i], pl.q[active[i]], tau, i == 0 ? s : P.side[i - 1]);
        if (e != cudaSuccess) return e;
    }
    for (int i = 1; i < na; ++i) {
        e = cudaEventRecord(P.join[i - 1], P.side[i - 1]);
        if (e != cudaSuccess) return e;
        e = cudaStreamWaitEvent(s, P.join[i - 1], 0);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

JPlanSet* jplan_create(const std::vector<int2> (&tiles)[kClasses][kClasses], const std::vector<int>& frag_npp,
                       const std::vector<int>& pair_x, const std::vector<int>& pair_y, int device)
{
    JPlanSet* P = new JPlanSet();
    for (int LP = 0; LP < kClasses; ++LP)
        for (int LQ = 0; LQ < kClasses; ++LQ) {
            const int cls = LP * kClasses + LQ;
            P->tiles[cls] = tiles[LP][LQ];
            P->nk[cls].resize(tiles[LP][LQ].size());
            for (size_t i = 0; i < tiles[LP][LQ].size(); ++i) {
                const int2 t = tiles[LP][LQ][i];
                const int pr = t.x >> 1;
                const int ky = (t.x & 1) ? pair_x[pr] : pair_y[pr];
                P->nk[cls][i] = frag_npp[ky * kClasses + LQ];
            }
        }
    cudaDeviceGetAttribute(&P->n_sm, cudaDevAttrMultiProcessorCount, device);
    for (auto& st : P->side) cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&P->fork, cudaEventDisableTiming);
    for (auto& e : P->join) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    cudaEventCreate(&P->t0);
    cudaEventCreate(&P->t1);
    // defaults: persistent queues for the FP64 core; for the FP32 and float-float cores, whose merged
    // persistent kernels carry the largest class's register footprint, the class kernels launched
    // concurrently on three streams (measured fastest for both on the water workloads)
    P->plan[1].persistent = 2;
    P->plan[2].persistent = 2;
    // ket chunks of the register classes on small workloads: a class whose whole-range work items give
    // fewer than 32 warps per SM is cut into 64-pair ket chunks, so that its launch balances over the
    // SMs instead of ending on a partial wave (64 waters: FP32 0.53 -> 0.48 ms, FP64 11.6 -> 11.5 ms per
    // build; 500 waters: whole ranges fastest)
    for (int cls = 0; cls < kNumCls; ++cls) {
        const int LP = cls / kClasses, LQ = cls % kClasses;
        if (LP + LQ >= 5 || P->tiles[cls].empty()) continue;
        int max_nk = 0;
        for (int v : P->nk[cls]) max_nk = std::max(max_nk, v);
        if (max_nk <= kSmallChunk) continue;
        const long long items = (long long)P->tiles[cls].size();
        const long long warps32 = LP <= 1 ? (items + 1) / 2 : items;  // two tiles per warp in the FP32 core
        if (items < 32LL * P->n_sm) P->plan[0].chunk[cls] = kSmallChunk;
        if (warps32 < 32LL * P->n_sm) P->plan[1].chunk[cls] = kSmallChunk;
    }
    return P;
}

void jplan_destroy(JPlanSet* P) { delete P; }

cudaError_t jplan_prepare(JPlanSet* P, int mode, cudaStream_t s)
{
    if (P->plan[mode].built) return cudaSuccess;
    return upload_plan(*P, mode, 1, s);
}

namespace {

// Strategy 2: the per-class kernels on the context stream and the two side streams, each class on
// the stream with the least work so far, classes in decreasing order of their estimated cost; the
// plan's ket chunk of a class cuts its tiles into shorter work items (more warps per launch).
cudaError_t launch_concurrent(JPlanSet& P, const Dev& d, int mode, const int2* tiles[kClasses][kClasses],
                              const int* n_tiles, float tau, cudaStream_t s)
{
    std::vector<std::pair<double, int>> cls;
    for (int c = 0; c < kNumCls; ++c) {
        if (n_tiles[c] <= 0) continue;
        double w = 0.0;
        for (int v : P.nk[c]) w += 32.0 * v * quartet_flops(c / kClasses, c % kClasses);
        cls.push_back({w, c});
    }
    if (cls.empty()) return cudaSuccess;
    std::stable_sort(cls.begin(), cls.end(), [](const std::pair<double, int>& a, const std::pair<double, int>& b) {
        return a.first > b.first;
    });
    cudaStream_t st[3] = {s, P.side[0], P.side[1]};
    double load[3] = {0.0, 0.0, 0.0};
    cudaError_t e = cudaEventRecord(P.fork, s);
    for (int i = 1; i < 3 && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(st[i], P.fork, 0);
    for (const auto& wc : cls) {
        if (e != cudaSuccess) break;
        int k = 0;
        for (int i = 1; i < 3; ++i)
            if (load[i] < load[k]) k = i;
        load[k] += wc.first;
        const int LP = wc.second / kClasses, LQ = wc.second % kClasses;
        const int chunk = P.plan[mode].chunk[wc.second];
        int nchunk = 1;
        if (chunk > 0)
            for (int v : P.nk[wc.second]) nchunk = std::max(nchunk, (v + chunk - 1) / chunk);
        e = launch_jengine_class(d, LP, LQ, tiles[LP][LQ], n_tiles[wc.second], tau, mode, st[k], chunk, nchunk);
    }
    for (int i = 1; i < 3 && e == cudaSuccess; ++i) {
        e = cudaEventRecord(P.join[i - 1], st[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, P.join[i - 1], 0);
    }
    return e;
}

}  // namespace

cudaError_t jplan_launch(JPlanSet* P, const Dev& d, int mode, const int2* tiles[kClasses][kClasses],
                         const int* n_tiles, double tau, cudaStream_t s)
{
    Plan& pl = P->plan[mode];
    if (pl.persistent == 2) return launch_concurrent(*P, d, mode, tiles, n_tiles, (float)tau, s);
    if (!pl.persistent || !pl.built) return launch_jengine(d, tiles, n_tiles, tau, mode, s);
    return launch_persistent(*P, d, mode, (float)tau, s);
}

void jplan_get(const JPlanSet* P, int mode, fef_tile_plan* out)
{
    const Plan& pl = P->plan[mode];
    out->persistent = pl.persistent;
    for (int i = 0; i < kNumCls; ++i) out->ket_chunk[i] = pl.chunk[i];
    out->tuned_ms = pl.tuned_ms;
}

cudaError_t jplan_set(JPlanSet* P, int mode, const fef_tile_plan* in, cudaStream_t s)
{
    Plan& pl = P->plan[mode];
    pl.persistent = std::min(2, std::max(0, in->persistent));
    for (int i = 0; i < kNumCls; ++i) pl.chunk[i] = std::max(0, in->ket_chunk[i]);
    pl.tuned_ms = in->tuned_ms;
    return upload_plan(*P, mode, 1, s);
}

namespace {

// Device time (ms) of one J-engine pass of the current plan of `mode` (best of reps after one
// warm-up); the accumulators receive garbage, so this runs only between builds.  The pass is captured
// into a CUDA graph on a private stream (ordered after s) and the graph is replayed: fef_iterate runs
// its builds as graph launches, where the per-kernel launch cost of the multi-stream plans is gone,
// so eager timing would favour the single-launch plans on small workloads.
cudaError_t time_plan(JPlanSet& P, const Dev& d, int mode, const int2* tiles[kClasses][kClasses],
                      const int* n_tiles, double tau, int reps, cudaStream_t s, double* ms)
{
    cudaStream_t cs = nullptr;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventRecord(P.t0, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, P.t0, 0);
    long long n_launch = 0;
    if (e == cudaSuccess) {
        const long long l0 = launches_so_far();
        // relaxed: the launchers set kernel attributes (cudaFuncSetAttribute) while capturing
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            const cudaError_t el = jplan_launch(&P, d, mode, tiles, n_tiles, tau, cs);
            const cudaError_t ec = cudaStreamEndCapture(cs, &g);  // ends the capture also after an error
            e = el != cudaSuccess ? el : ec;
        }
        n_launch = launches_so_far() - l0;
        note_launches(-n_launch);  // nothing ran during the capture
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
    double best = 1e300;
    for (int r = -1; r < reps && e == cudaSuccess; ++r) {
        e = cudaEventRecord(P.t0, cs);
        if (e == cudaSuccess) e = cudaGraphLaunch(ge, cs);
        if (e == cudaSuccess) note_launches(n_launch);
        if (e == cudaSuccess) e = cudaEventRecord(P.t1, cs);
        if (e == cudaSuccess) e = cudaEventSynchronize(P.t1);
        float f = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&f, P.t0, P.t1);
        if (e == cudaSuccess && r >= 0) best = std::min(best, (double)f);
    }
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    if (cs) {
        cudaStreamSynchronize(cs);
        cudaStreamDestroy(cs);
    }
    if (e != cudaSuccess) return e;
    *ms = best;
    return cudaSuccess;
}

}  // namespace

cudaError_t jplan_autotune(JPlanSet* P, const Dev& d, int mode, const int2* tiles[kClasses][kClasses],
                           const int* n_tiles, double tau, int reps, double budget_ms, cudaStream_t s,
                           fef_tile_plan* out)
{
    Plan& pl = P->plan[mode];
    reps = std::max(1, reps);
    double total_flops = 0.0;
    double cls_cost[kNumCls] = {};
    for (int cls = 0; cls < kNumCls; ++cls) {
        for (int v : P->nk[cls]) cls_cost[cls] += 32.0 * v * quartet_flops(cls / kClasses, cls % kClasses);
        total_flops += cls_cost[cls];
    }
    const double rate = mode == 1 ? 2e13 : (mode == 2 ? 2e12 : 5e11);  // flop/s
    const double est_ms = 1e3 * total_flops / rate;
    const bool full_passes = est_ms * 2 * (reps + 1) <= budget_ms;
    cudaError_t e = cudaSuccess;
    // 0. the plan in place (the default, or one the caller set) is a candidate too: when full passes
    //    fit the budget it is timed first and kept unless the tuned plan is faster
    const int start_persistent = pl.persistent;
    int start_chunk[kNumCls];
    std::copy(pl.chunk, pl.chunk + kNumCls, start_chunk);
    double t_start = -1.0;
    if (full_passes) {
        e = upload_plan(*P, mode, 1, s);
        if (e == cudaSuccess) e = time_plan(*P, d, mode, tiles, n_tiles, tau, reps, s, &t_start);
        if (e != cudaSuccess) return e;
    }
    // 1. default persistent plan; the tuning passes run on every stride-th fragment pair so that one
    //    pass takes about budget/64 (estimated from the flop count at a conservative rate)
    pl.persistent = 1;
    for (int i = 0; i < kNumCls; ++i) pl.chunk[i] = 0;
    const double per_pass = std::max(1.0, budget_ms / 64.0);
    const int stride = std::max(1, (int)std::ceil(est_ms / per_pass));
    // 2. per class pair, in decreasing order of its share of the estimated cost, the ket chunk
    std::vector<int> order(kNumCls);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cls_cost[a] > cls_cost[b]; });
    if (stride > 1) {
        e = upload_plan(*P, mode, stride, s);
        if (e != cudaSuccess) return e;
    }
    double best = 0.0;
    e = time_plan(*P, d, mode, tiles, n_tiles, tau, reps, s, &best);
    if (e != cudaSuccess) return e;
    for (int cls : order) {
        if (cls_cost[cls] <= 0.0) continue;
        int max_nk = 0;
        for (int v : P->nk[cls]) max_nk = std::max(max_nk, v);
        const int keep = pl.chunk[cls];
        int best_c = keep;
        for (int c : kChunkCandidates) {
            if (c == keep || (c > 0 && c >= max_nk)) continue;  // same items as the whole range
            pl.chunk[cls] = c;
            e = upload_plan(*P, mode, stride, s);
            if (e != cudaSuccess) return e;
            double t = 0.0;
            e = time_plan(*P, d, mode, tiles, n_tiles, tau, reps, s, &t);
            if (e != cudaSuccess) return e;
            if (t < best * 0.99) {
                best = t;
                best_c = c;
            }
        }
        pl.chunk[cls] = best_c;
    }
    // 3. the chosen chunks on the full workload, against one launch per class pair when a full pass
    //    fits the budget
    e = upload_plan(*P, mode, 1, s);
    if (e != cudaSuccess) return e;
    pl.tuned_ms = best * stride;  // estimate from the sample
    if (full_passes) {
        double t_pers = 0.0, t_leg = 0.0;
        e = time_plan(*P, d, mode, tiles, n_tiles, tau, reps, s, &t_pers);
        if (e != cudaSuccess) return e;
        double t_conc = 0.0;
        pl.persistent = 0;
        e = time_plan(*P, d, mode, tiles, n_tiles, tau, reps, s, &t_leg);
        if (e != cudaSuccess) return e;
        pl.persistent = 2;
        e = time_plan(*P, d, mode, tiles, n_tiles, tau, reps, s, &t_conc);
        if (e != cudaSuccess) return e;
        pl.persistent = 1;
        pl.tuned_ms = t_pers;
        if (t_leg < pl.tuned_ms) {
            pl.persistent = 0;
            pl.tuned_ms = t_leg;
        }
        if (t_conc < pl.tuned_ms) {
            pl.persistent = 2;
            pl.tuned_ms = t_conc;
        }
        if (t_start > 0.0 && t_start <= pl.tuned_ms) {
            pl.persistent = start_persistent;
            std::copy(start_chunk, start_chunk + kNumCls, pl.chunk);
            pl.tuned_ms = t_start;
        }
        // the work queues of the plan kept (its ket chunks may be the starting plan's)
        e = upload_plan(*P, mode, 1, s);
        if (e != cudaSuccess) return e;
    }
    if (out) jplan_get(P, mode, out);
    return cudaSuccess;
}

}  // namespace fef
