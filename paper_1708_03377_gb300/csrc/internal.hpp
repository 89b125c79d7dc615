// Internal data layout of a FEF context in device memory, and the kernel launchers shared by the
// translation units of libfef.so.  Not part of the public ABI (include/fef.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/fef.h"

namespace fef {

constexpr int kClasses = 5;  // Hermite class L_P = l_a + l_b = 0..4

// Structure-of-arrays views of everything the kernels read.  All pointers are device pointers.
//   atoms  : xyz in bohr, Z as double
//   shells : l, primitive count/offset, AO offset inside the fragment, owning atom and fragment
//   prims  : exponent, coefficient times the shell-level normalisation (2a/pi)^{3/4} (4a)^{l/2}
//   AOs    : ao_scale (unit self-overlap), indexed by global AO = frag_ao0[x] + local AO
//   shell pairs (a <= b inside one fragment): class L, first primitive pair in its class array,
//            Schwarz factor Q_ab
//   primitive pairs, per class L: centre P and exponent p (double4_32a), FP32 copy (float4),
//            K = c_i c_j exp(-a b/p |AB|^2), shell-pair id, primitive indices, Schwarz factor (float),
//            Hermite density Dh[nh(L)][n] and Hermite Coulomb accumulator Jh[nh(L)][n] (SoA)
//   packed matrices: per fragment a full n_x*n_x row-major block at frag_moff[x]
struct Dev {
    int n_frag, n_atoms, n_shells, n_sp, n_pairs;
    int max_nao;
    int max_l;  // largest shell angular momentum
    // atoms
    const double* atom_xyz;
    const double* atom_Z;
    // fragments
    const int* frag_atom0;
    const int* frag_nat;
    const int* frag_sh0;
    const int* frag_nsh;
    const int* frag_nao;
    const int* frag_ao0;
    const int* frag_sp0;
    const int* frag_nocc;
    const int64_t* frag_moff;
    const int64_t* frag_eoff;
    const int64_t* frag_coff;  // packed Coulomb-minus-half-exchange tensor, (n(n+1)/2)^2 per fragment
    const int* frag_pp0;   // [n_frag*kClasses] first prim pair of class L in the class array
    const int* frag_npp;   // [n_frag*kClasses]
    const int* frag_nbr0;  // [n_frag+1] CSR neighbour list
    const int* nbr;        // neighbour fragment ids
    const int* nbr_pair;   // pair index of each CSR entry
    // shells / prims / AOs
    const int* sh_l;
    const int* sh_np;
    const int* sh_p0;
    const int* sh_ao;
    const int* sh_atom;
    const double* p_exp;
    const double* p_coef;
    const double* ao_scale;
    const int* ao_sh;      // [n_ao_total] global shell of each AO
    const int* ao_k;       // [n_ao_total] Cartesian component inside its shell
    // shell pairs
    const int* sp_a;
    const int* sp_b;
    const int* sp_L;
    const int* sp_pp0;
    const double* sp_Q;
    // primitive pairs per class
    const double4_32a* pp_P[kClasses];
    const float4* pp_Pf[kClasses];
    const double* pp_K[kClasses];
    const int* pp_sp[kClasses];
    const int* pp_ij[kClasses];  // i * 16 + j
    const float* pp_Q[kClasses];
    double* pp_Dh[kClasses];
    double* pp_Jh[kClasses];
    const float4* pp_Pr[kClasses];   // FP32 (P - anchor of the fragment, p) for the mixed J-engine
    float* pp_Dh32[kClasses];        // FP32 scratch of nh(L) floats per pair (learned-start descriptors)
    const double* pp_rp[kClasses];   // p^{-1/2} per primitive pair (asymptotic J-engine path)
    double* pp_u[kClasses];          // FP64 J-engine weights u = p^{-1/2} D_P (SoA like pp_Dh), per build
    const int* pp_perm[kClasses];    // bra order of the J-engine: each fragment's class range sorted by p
    float* pp_rec32[kClasses];       // FP32-core record per primitive pair (rec32_len(L) floats, see jengine.cu)
    const float* fc_qmin;            // [n_frag*kClasses] smallest Schwarz factor of each fragment's class
    const float4* pp_Phi[kClasses];  // df64 (P, p): high floats ...
    const float4* pp_Plo[kClasses];  // ... and low floats (float-float J-engine)
    float2* pp_udf[kClasses];        // df64 weights u = p^{-1/2} D_P (hi, lo), per float-float build
    const float2* pp_sqdf[kClasses]; // df64 sqrt(p)
    int n_pp[kClasses];
    // fragment pairs
    const int* pair_x;
    const int* pair_y;
    // tables / scratch
    const double* boys;
    const float* boys32;
    const float2* boysdf;            // df64 copy of the FP64 Boys table
    int* err_flag;
};

// FP32-core record of a primitive pair of class L, rebuilt for every FP32-core build (jengine.cu):
// (P - anchor of its fragment, p) | (k_hi, k_lo, Schwarz factor, 0) | u[0..nh(L)-1], padded to a
// multiple of 4 floats, with k = (sqrt(pi)/2) p^{-1/2} as a float pair and u = p^{-1/2} (D_P - D_P^ref).
__host__ __device__ constexpr int rec32_len(int L)
{
    return 8 + (((L + 1) * (L + 2) * (L + 3) / 6 + 3) & ~3);
}

// fragment owning shell pair s (frag_sp0 is ascending)
__device__ inline int frag_of_shellpair(const Dev& d, int s)
{
    int lo = 0, hi = d.n_frag - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (d.frag_sp0[mid] <= s) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Host-side context.
struct Buffers;
constexpr int kHistoryFields = 9;
}  // namespace fef

struct fef_ctx {
    fef_options opt;
    cudaStream_t stream = nullptr;
    int device = 0;
    int n_frag = 0, n_atoms = 0, n_shells = 0, n_prims = 0, n_sp = 0, n_pairs = 0;
    int n_nbr = 0;  // entries of the neighbour CSR list (2 n_pairs)
    int64_t mat_total = 0, eri_total = 0, coff_total = 0;
    int max_nao = 0, max_nmo = 0;
    std::vector<int> nao, nmo, nocc;
    std::vector<int64_t> moff;
    std::vector<int> h_pair_x, h_pair_y;
    std::vector<int> h_frag_sp0, h_sp_a, h_sp_b, h_sh_l;  // shell pairs (intra-ERI tasks of E_M2)
    std::vector<int> h_frag_pp0, h_frag_npp;              // [n_frag * 5] primitive-pair class ranges
    fef::Dev dev{};
    fef::Buffers* buf = nullptr;
    // counters
    int64_t shell_quartets = 0, prim_quartets = 0;
    int64_t class_quartets[25] = {};
    double jengine_ms = 0.0;
    // one record per macro-iteration of the last fef_iterate (index 0: the start densities):
    // k, E_tot, |dE_tot|, max|dE_x|, max micro-iterations, summed micro-iterations, J-engine ms, SCF ms,
    // 1 if the build used the FP32 core
    std::vector<double> history;
    bool have_density = false;
    bool last_build_fp32 = false;
    fef_mlp* warm_start = nullptr;  // network used when start = FEF_START_LEARNED (not owned)
    int learn_feat = 0, learn_pack = 0;  // 0: fragments not uniform or have d shells
    int learn_desc = 0;                  // potential/field part of the features (4 per atom)
    bool energies_valid = false;
    std::string last_error;
};

namespace fef {

// Number of kernels launched by this library since load (incremented at every launch site).
void note_launches(long long n);
long long launches_so_far();

// ---- kernels launched by the API layer (each returns cudaGetLastError()) ----
cudaError_t launch_prepare(const Dev& d, const double* xyz_A, double* atom_xyz, double* p_coef_out,
                           const double* p_coef_raw, const int* p_l, int n_prims, cudaStream_t s);
cudaError_t launch_boys_table(double* table, cudaStream_t s);
cudaError_t launch_ao_scale(const Dev& d, double* ao_scale, int n_ao_total, const int* ao_frag, cudaStream_t s);
cudaError_t launch_prim_pairs(const Dev& d, double4_32a* P[kClasses], float4* Pf[kClasses], double* K[kClasses],
                              float4* Pr[kClasses], double* rp[kClasses], cudaStream_t s);
// smallest Schwarz factor of each fragment's primitive pairs of each class (after launch_schwarz)
cudaError_t launch_class_qmin(const Dev& d, float* qmin, cudaStream_t s);
// FP32-core records of every class for the density difference D - D_ref (Hermite densities in pp_Dh,
// reference in Dh_ref, NULL entries = 0), with charge-conserving rounding of each fragment's u[0]
// (resid: workspace of max n_pp doubles)
cudaError_t launch_fp32_records(const Dev& d, double* const Dh_ref[kClasses], double* resid, cudaStream_t s);
cudaError_t launch_boys_table32(const double* table64, float* table32, cudaStream_t s);
// Dh32 = float(Dh - Dh_ref) for every class
cudaError_t launch_one_electron(const Dev& d, double* S, double* h, cudaStream_t s);
// far field (pairs beyond the cutoff): moment integrals about each fragment's centroid (10 n^2 at
// 10 frag_moff), per build the fragments' multipoles, the far potentials and the Fock/omega terms,
// and the energies (E_frag += E_far, E_tot recomputed)
cudaError_t launch_moment_integrals(const Dev& d, const double* cen, double* M, cudaStream_t s);
cudaError_t launch_far_field(const Dev& d, const double* M, const double* Mnuc, const double* cen, const double* D,
                             double* mult, double* pot, double* E_far, double* F, double* omega, cudaStream_t s);
cudaError_t launch_far_energy(const Dev& d, const double* E_far, double* E_frag, double* E_tot, cudaStream_t s);
// The same multipole expansion over the neighbours within the cutoff: omega (n_omega doubles, zeroed
// first) = -(phi S + grad phi . <r> + (1/2) hess phi : <r r>) of each fragment's neighbours' multipoles
// for the densities D (the learned start's estimate of the environment operator, no Fock build).
cudaError_t launch_near_multipole_field(const Dev& d, const double* M, const double* Mnuc, const double* cen,
                                       const double* D, double* mult, double* pot, double* omega, int64_t n_omega,
                                       cudaStream_t s);
// Bra components per task of the specialised s/p intra-fragment ERI kernels: consecutive components
// kb0 .. kb0 + NKB - 1 share each primitive quartet's Boys values and R recursion, as many as fit in
// registers beside the bra's Hermite tables (all components when at most 27 outputs and no p-p bra
// pair; for a p-p bra pair one Cartesian row against an s or p ket component set of at most 3, else
// one component).  Tasks of classes with a d shell take one component each.
__host__ __device__ constexpr int intra_nkb(int la, int lb, int lc, int ld)
{
    return (la > 1 || lb > 1 || lc > 1 || ld > 1) ? 1
           : (la == 1 && lb == 1) ? ((1 + 2 * lc) * (1 + 2 * ld) <= 3 ? (lc + ld == 0 ? 9 : 3) : 1)
           : ((1 + 2 * la) * (1 + 2 * lb) * (1 + 2 * lc) * (1 + 2 * ld) <= 27 ? (1 + 2 * la) * (1 + 2 * lb) : 1);
}

// intra-fragment ERI rows for tasks (fragment, shell pair s1, shell pair s2 >= s1, bra component) sorted
// by class cls = ((la 3 + lb) 3 + lc) 3 + ld, class c at [cls_off[c], cls_off[c + 1]) (intra_eri_tasks)
cudaError_t launch_intra_eri(const Dev& d, const int4* tasks, const std::vector<int>& cls_off, double* eri,
                             cudaStream_t s);
cudaError_t launch_schwarz(const Dev& d, const double* eri, double* sp_Q, float* pp_Q[kClasses], cudaStream_t s);
cudaError_t launch_coulomb_exchange(const Dev& d, const double* eri, double* eric, cudaStream_t s);
cudaError_t launch_neighbours(const Dev& d, double cutoff_bohr, unsigned char* flags, cudaStream_t s);
cudaError_t launch_nuclear_env(const Dev& d, double* vh[kClasses], double* V, cudaStream_t s);
// Hermite fields of each pair's nuclei on the other member's primitive pairs (geometry time), and
// per build tr[D^x V^y] per pair and direction as their dot product with the Hermite densities.
cudaError_t launch_nuclear_trace_fields(const Dev& d, const int64_t* off, double* fields, cudaStream_t s);
cudaError_t launch_nuclear_traces(const Dev& d, const int64_t* off, const double* fields, double* trace_xy,
                                  double* trace_yx, cudaStream_t s);
cudaError_t launch_nuclear_repulsion(const Dev& d, double* e_nn_intra, double* e_nn_pair, cudaStream_t s);
// X = U s^{-1/2} (canonical); optionally S^{1/2} and S^{-1/2} (symmetric) into Sh, Sih
cudaError_t launch_orthogonaliser(const Dev& d, const double* S, double* X, int* nmo, double s_min, int max_n,
                                  cudaStream_t s, double* Sh = nullptr, double* Sih = nullptr,
                                  double* ws = nullptr);
cudaError_t launch_hermite_density(const Dev& d, const double* D, cudaStream_t s);
// mode 0: FP64 J-engine on pp_Dh; mode 1: FP32-core J-engine on the FP32 records; mode 2: float-float
// J-engine on pp_udf for the s/p classes, FP64 for the rest.  All add into the FP64 accumulators
// pp_Jh.
cudaError_t launch_jengine(const Dev& d, const int2* tiles[kClasses][kClasses], const int* n_tiles, double tau,
                           int mode, cudaStream_t s);
cudaError_t launch_jengine_df(const Dev& d, const int2* tiles[kClasses][kClasses], const int* n_tiles, float tau,
                              cudaStream_t s);
// one class pair's per-class kernel (mode as launch_jengine), for concurrent launches on forked streams;
// chunk > 0 (register classes): each tile's ket range cut into nchunk chunks of chunk pairs
cudaError_t launch_jengine_class(const Dev& d, int LP, int LQ, const int2* t, int n, float tau, int mode,
                                 cudaStream_t s, int chunk = 0, int nchunk = 1);
cudaError_t launch_jengine_big_class(const Dev& d, int LP, int LQ, const int2* t, int n, float tau, int fp32,
                                     cudaStream_t s);
cudaError_t launch_jengine_df_class(const Dev& d, int LP, int LQ, const int2* t, int n, float tau, cudaStream_t s);
cudaError_t launch_df_setup(const Dev& d, float4* const Phi[kClasses], float4* const Plo[kClasses],
                            float2* const sqdf[kClasses], float2* boysdf, cudaStream_t s);
cudaError_t launch_df_density(const Dev& d, cudaStream_t s);
cudaError_t launch_jengine_big(const Dev& d, const int2* tiles[kClasses][kClasses], const int* n_tiles, float tau,
                               int fp32, cudaStream_t s);
// Persistent J-engine (one launch per register tier and Fock build, warps take cost-sorted work
// items from a queue).  Item (int4): x = 2 pair + swap, y = first bra primitive pair of the 32-pair
// tile, z = first ket pair and (w >> 5) = end ket pair, both as offsets in the partner fragment's
// class-LQ range, (w & 31) = LP * kClasses + LQ.
constexpr int kItemClassBits = 5;
__host__ __device__ inline int jitem_class(int4 it) { return it.w & ((1 << kItemClassBits) - 1); }
__host__ __device__ inline int jitem_ket_end(int4 it) { return it.w >> kItemClassBits; }
struct JQueue {
    const int4* items = nullptr;  // device, sorted by decreasing estimated cost
    int n = 0;
    int* next = nullptr;          // device counter, zeroed by the launcher before every launch
    int grid = 0;                 // resident blocks of the kernel on this device
    int smem_slice = 0;           // shared-memory R tier: Reals per warp (largest class of the queue)
};
// MODE 0 FP64, 1 FP32 core; spd: the queue holds register classes with L_P >= 3
cudaError_t jengine_persistent_grid(int mode, bool spd, int* blocks_per_sm);
cudaError_t launch_jengine_persistent(const Dev& d, int mode, bool spd, const JQueue& q, float tau, cudaStream_t s);
// float-float core for the s/p classes (L_P <= 2)
cudaError_t jengine_df_persistent_grid(int* blocks_per_sm);
cudaError_t launch_jengine_df_persistent(const Dev& d, const JQueue& q, float tau, cudaStream_t s);
// classes with L_P + L_Q >= 5 (R in shared memory); fp32 selects the FP32 core
int jengine_big_slice(int LP, int LQ);
cudaError_t jengine_big_persistent_grid(int fp32, int smem_slice, int* blocks_per_sm);
cudaError_t launch_jengine_big_persistent(const Dev& d, int fp32, const JQueue& q, float tau, cudaStream_t s);
// Tile plans of the J-engine (jplan.cu): per engine mode (0 FP64, 1 FP32 core, 2 float-float) the
// strategy (persistent queues or one launch per class pair) and the ket chunk per class pair.
struct JPlanSet;
JPlanSet* jplan_create(const std::vector<int2> (&tiles)[kClasses][kClasses], const std::vector<int>& frag_npp,
                       const std::vector<int>& pair_x, const std::vector<int>& pair_y, int device);
void jplan_destroy(JPlanSet* P);
cudaError_t jplan_prepare(JPlanSet* P, int mode, cudaStream_t s);  // build the queues (not while capturing)
cudaError_t jplan_launch(JPlanSet* P, const Dev& d, int mode, const int2* tiles[kClasses][kClasses],
                         const int* n_tiles, double tau, cudaStream_t s);
void jplan_get(const JPlanSet* P, int mode, fef_tile_plan* out);
cudaError_t jplan_set(JPlanSet* P, int mode, const fef_tile_plan* in, cudaStream_t s);
cudaError_t jplan_autotune(JPlanSet* P, const Dev& d, int mode, const int2* tiles[kClasses][kClasses],
                           const int* n_tiles, double tau, int reps, double budget_ms, cudaStream_t s,
                           fef_tile_plan* out);
cudaError_t launch_back_transform(const Dev& d, double* J, cudaStream_t s);
// F = h + C D + V_env + J_env per fragment; E_int[x] = tr[D (h + G/2)] + e_nn[x]; tr_omega[x] = tr[D (V+J)]
// also trV[x] = tr(D^x V_env^x), trJ[x] = tr(D^x J_env^x)
cudaError_t launch_fock_energy(const Dev& d, const double* h, const double* Venv, const double* Jenv,
                               const double* eric, const double* D, double* F, double* omega, const double* e_nn,
                               double* E_int, double* trV, double* trJ, cudaStream_t s);
cudaError_t launch_count_quartets(const Dev& d, double tau, unsigned long long* count, cudaStream_t s);

struct ScfArgs {
    const double* h;        // packed
    const double* omega;    // packed environment field (may be null: isolated)
    const double* S;
    const double* X;
    const int* nmo;
    const double* eric;     // eric_packed = 0: full C[mu nu][lambda sigma], n^4 at frag_eoff;
                            // eric_packed = 1: packed transposed CT[rs][pq] at frag_coff (see setup.cu)
    int eric_packed;
    const double* e_nn;     // [n_frag] own nuclear repulsion
    double* D;              // in: start (if have_start), out: converged
    double* F;              // out: Fock of the returned D
    double* diis_F;         // scratch [n_frag][diis][n^2]
    double* diis_e;         // scratch [n_frag][diis][n^2]
    int64_t diis_stride;    // per fragment doubles
    double* E_scf;          // [n_frag]
    double* E_int;          // [n_frag]
    int* iters;             // [n_frag]
    int have_start;
    int max_iter, diis_size;
    double e_tol, comm_tol;
    double* ws;             // global workspace, 9 n^2 doubles per fragment at 9 frag_moff[x]: used by
                            // fragments above kScfSmemMaxN AOs (null when there are none)
    int diis_by_moff;       // 1: DIIS history at 2 diis_size frag_moff[x] (sized per fragment),
                            // 0: at x * diis_stride
    const int* list;        // fragments of the one-block-per-fragment launch (null: all fragments)
    int n_list;
    double* gap;            // [n_frag] HOMO-LUMO gap of the last Roothaan step (nullable)
    const double* tol;      // device [2]: e_tol, comm_tol of this launch (null: the fields above)
    int shift_after;        // > 0: from micro-iteration shift_after + 1 on, level shift the virtual
    double level_shift;     // orbitals by level_shift (hartree) and restart DIIS (0: never)
    const int* big_list;    // fragments above kScfSmemMaxN AOs, one thread-block cluster each
    int n_big;              // (0: none; then list is null or holds every fragment)
};
cudaError_t launch_fragment_scf(const Dev& d, const ScfArgs& a, int max_n, cudaStream_t s);

// E_M2 (Eq. EM2) per fragment, one block per fragment (any size up to kMaxFragAO): canonical orbitals of
// F (packed), (ia|jb) by four quarter-transforms of the pair-packed U, closed-shell second-order sum.
int64_t energy_m2_workspace(int n, int nocc, int nmo);  // doubles per fragment
// E_D2 (Eq. ED2): canonical orbitals (C packed at frag_moff, eps at frag_ao0; Jacobi workspace
// 2 frag_moff), inter-fragment pair blocks W (k_pair_eri), per-pair transform and second-order sum
cudaError_t launch_canonical_orbitals(const Dev& d, const double* F, const double* X, const int* nmo, double* ws,
                                      double* C, double* eps, cudaStream_t s);
cudaError_t launch_pair_eri(const Dev& d, const int4* tasks, int n_tasks, const int* pair_of, const int64_t* off,
                            double* W, cudaStream_t s);
int64_t energy_d2_workspace(int nx, int ox, int mx, int ny, int oy, int my);  // doubles per pair
cudaError_t launch_energy_d2(const Dev& d, int n_pairs, const int* pair_of, const int64_t* woff, const double* W,
                             const double* C, const double* eps, const int* nmo, const int64_t* toff, double* tws,
                             double* E, cudaStream_t s);
// E_D2 on transition Hermite densities (ed2.cu; fragments with s and p shells): U = per fragment the
// pre-scaled Hermite transition densities of all occupied-virtual pairs, rows (class offset hoff, local
// primitive pair, Hermite component) x columns ov; per chunk of pairs the fields G of the partner's
// transition densities on each bra primitive pair (items per bra class: 2 q + side, first bra pair,
// first column), then E_D2 per pair as ed2_energy_slices(max_entries) partial sums per pair
// (E[q * slices + k], max_entries = the chunk's largest n_ov(x) n_ov(y)).
cudaError_t launch_ed2_transition(const Dev& d, const double* C, const int* nmo, const int64_t* uoff, const int* hoff,
                                  const int* n_ov, int max_ov, double* U, cudaStream_t s);
cudaError_t launch_ed2_split(const double* U, float2* Udf, int64_t n, cudaStream_t s);  // float-float copy of U
cudaError_t launch_ed2_pairs(const Dev& d, const double* U, const float2* Udf, const int64_t* uoff, const int* hoff,
                             const int* n_ov, const int* pair_of, const int64_t* goff, double* G, double tau,
                             const int4* const items[3], const int n_items[3], cudaStream_t s);
cudaError_t launch_ed2_energy(const Dev& d, int n_pairs, int max_entries, const double* U, const int64_t* uoff,
                              const int* hoff, const int* n_ov, const int* pair_of, const int64_t* goff, const double* G,
                              const double* C, const double* eps, const int* nmo, const int* n_herm, double* E,
                              cudaStream_t s);
int ed2_cols_per_item(int LB);
int ed2_energy_slices(int max_entries);
cudaError_t launch_energy_m2(const Dev& d, const double* F, const double* X, const int* nmo, const double* U,
                             const int64_t* ws_off, double* ws, double* E, cudaStream_t s);

// E_frag[x] = E_int[x] + (trV[x] + sum_y tr(D^y V^x) + trJ[x] + sum_y E_nn(x,y)) / 2, E_tot = sum E_frag
cudaError_t launch_energies(const Dev& d, const double* E_int, const double* trV, const double* trJ,
                            const double* tr_xy, const double* tr_yx, const double* e_nn_pair, double* E_frag,
                            double* E_tot, cudaStream_t s);
cudaError_t launch_check_finite(const double* a, int64_t n, int* flag, cudaStream_t s);

cudaError_t measure_fma_peak(double* fp64, double* fp32, double* mhz);

// learned warm start (learned.cu, mlp.cu)
cudaError_t launch_frames(const Dev& d, double* rot, cudaStream_t s);
// descriptors: part holds n_nbr * max_nat * 4 doubles (per neighbour entry and atom)
cudaError_t launch_descriptors(const Dev& d, const double* rot, int n_feat, int max_nat, int n_nbr, double* part,
                               float* X, cudaStream_t s);
cudaError_t launch_local_density(const Dev& d, const double* rot, const double* Sh, const double* D, int stride,
                                 int col0, float* out, cudaStream_t s);
cudaError_t launch_apply_learned(const Dev& d, const double* rot, const double* Sih, const double* D_iso,
                                 const float* dloc, int n_pack, double* D, cudaStream_t s);
cudaError_t mlp_predict_device(fef_mlp* m, const float* X, float* Y, int n, cudaStream_t st);
int mlp_n_in(const fef_mlp* m);
int mlp_n_out(const fef_mlp* m);

}  // namespace fef
