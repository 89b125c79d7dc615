/*
 * fef.h - C ABI of the GB300 fragment-effective-field (FEF) mean-field library (libfef.so).
 *
 * The method is the polarization-screened fragment mean field of Byrd, Molt, Bartlett & Sanders
 * (arXiv:1708.03377), Theory section, "Fragment Mean Field":
 *
 *   - the system is split into fragments x, each with its own monomer-centred AO basis and its own
 *     closed-shell determinant (product ansatz with the antisymmetriser dropped, Eq. prodspace);
 *   - each fragment's Fock matrix is F~ = h(1) + (2J - K) + omega_x; in AO form, with
 *     D^x = 2 C_occ C_occ^T,  F^x = h^x + G[D^x] + omega_x,  G[D] = J[D] - K[D]/2;
 *   - omega_x = h~ + 2 v (Eq. wc): h~ is the attraction of x's electrons to the nuclei of every other
 *     fragment y and 2 v (Eq. dp2e) is the Coulomb matrix of y's density,
 *     J[D^y]_{mu nu} = sum_{lambda sigma in y} (mu nu|lambda sigma) D^y_{lambda sigma};
 *     there is no inter-fragment exchange;
 *   - the field is relaxed to all orders (the polarisation-screened mean field): every fragment's
 *     RHF is solved in the field of the others and the field rebuilt until all fragments are
 *     self-consistent.
 *
 * Conventions used by every call:
 *   - Units: geometry in Angstrom on input (1 bohr = 0.529177210903 A); bohr and hartree inside
 *     and on output.
 *   - Basis: contracted Cartesian Gaussians, l = 0 (s), 1 (p), 2 (d), Cartesian components of a
 *     shell in lexicographic order (x, y, z; xx, xy, xz, yy, yz, zz).  A raw contraction
 *     coefficient multiplies a primitive normalised at shell level, (2a/pi)^{3/4} (4a)^{l/2}
 *     x^lx y^ly z^lz exp(-a r^2); every Cartesian AO is then renormalised to unit self-overlap.
 *     Shells of an atom come in the order of its basis set; AOs of a fragment follow its atoms.
 *   - Matrix layout: "packed" = for each fragment x in order, the full n_x-by-n_x row-major block,
 *     blocks concatenated (offsets from fef_ao_layout).
 *   - Pointers: host pointers unless a call's on_device flag is 1, in which case they are device
 *     pointers in the current CUDA context, used on the context's stream.  Inputs are copied
 *     during the call; outputs are caller-allocated.  All device work of a context runs on the
 *     stream given to fef_create (NULL = the legacy default stream); every call that returns host
 *     data synchronises that stream before returning.
 *   - Errors: every call returns a fef_status; fef_last_error gives a message for the last failing
 *     call on the context.  No exception crosses the ABI.  A context stays valid after
 *     FEF_ERR_NOT_CONVERGED.  A context is used by one host thread at a time.
 */
#ifndef FEF_H
#define FEF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fef_ctx fef_ctx;

typedef enum {
    FEF_OK = 0,
    FEF_ERR_ARG = 1,            /* invalid argument, size or pointer */
    FEF_ERR_BASIS = 2,          /* bad exponents / l > 2 / linearly dependent fragment basis */
    FEF_ERR_GEOM = 3,           /* odd electron count, coincident atoms, bad fragment map */
    FEF_ERR_CUDA = 4,           /* a CUDA call failed; message has the CUDA error string */
    FEF_ERR_NOT_CONVERGED = 5,  /* SCF or FEF iteration hit its iteration limit */
    FEF_ERR_NUMERIC = 6         /* NaN/Inf met in a Fock matrix, density or energy */
} fef_status;

enum { FEF_FP64 = 0, FEF_MIXED = 1 };
enum { FEF_ENGINE_FP64 = 0, FEF_ENGINE_DF64 = 1 };
enum { FEF_START_SUPERPOSITION = 0, FEF_START_LEARNED = 1, FEF_START_GIVEN = 2 };
enum { FEF_MIXED_INCREMENT = 0, FEF_MIXED_WHOLE = 1 };

/* Molecular system split into fragments (Theory, "Fragment Mean Field": Hilbert space partition
 * into fragment subspaces, monomer-centred basis). */
typedef struct {
    int32_t n_atoms;
    const int32_t* Z;              /* [n_atoms] nuclear charges, 1..36 */
    const double* xyz;             /* [n_atoms*3] Angstrom */
    const int32_t* frag_of_atom;   /* [n_atoms] fragment index; each fragment a contiguous run, in order */
    const int32_t* basis_of_atom;  /* [n_atoms] index of the atom's basis set in fef_basis */
    int32_t n_frag;
    const int32_t* charge;         /* [n_frag] net charge, or NULL for all neutral */
} fef_geometry;

/* Basis sets: n_sets kinds; set k owns shells [set_shell_offset[k], set_shell_offset[k+1]). */
typedef struct {
    int32_t n_sets;
    const int32_t* set_shell_offset;  /* [n_sets+1] */
    const int32_t* shell_l;           /* [n_shells] 0, 1 or 2 */
    const int32_t* shell_nprim;       /* [n_shells] 1..8 */
    const double* exps;               /* [sum nprim] exponents > 0, shell after shell */
    const double* coefs;              /* [sum nprim] raw contraction coefficients */
} fef_basis;

typedef struct {
    int32_t precision;       /* FEF_FP64, or FEF_MIXED: fef_iterate's first field comes from the FP32-core
                                J-engine and becomes the reference D_ref; later builds add the FP32-core
                                J-engine of D - D_ref to the stored field of D_ref (FP64 accumulation,
                                FP64 intra-fragment G, eigensolve and energies) until |dE| <
                                mixed_switch (or stops decreasing); then one FP64 build becomes the
                                exact reference and FP32 increments relative to it continue to
                                convergence (from every start). */
    double cutoff_A;         /* fragment pairs with min atom-atom distance >= cutoff are dropped
                                (J and V together); <= 0 keeps all pairs */
    double schwarz;          /* shell quartet (ab|cd) dropped when Q_ab Q_cd < schwarz (0: none) */
    double e_tol;            /* FEF convergence: |dE_tot| < e_tol and max_x |dE_x| < e_tol */
    double micro_e_tol;      /* fragment RHF: |dE_x^scf| < micro_e_tol ... */
    double micro_comm_tol;   /* ... and max |F D S - S D F| < micro_comm_tol.  Inside fef_iterate these
                                are floors: each macro-iteration's fragment RHF stops at
                                max(floor, min(1e-7, 1e-5 dE)) and max(floor, min(1e-5, 1e-3 dE)),
                                dE the previous macro-iteration's energy change (1e-3 for the first) */
    int32_t max_macro;       /* FEF macro-iterations limit */
    int32_t max_micro;       /* fragment RHF iterations limit per macro-iteration */
    int32_t diis_size;       /* Pulay DIIS subspace size, 1..8 (1 = plain Roothaan) */
    int32_t start;           /* FEF_START_*: initial densities */
    int32_t use_graph;       /* 1 (default): each macro-iteration (fragment SCF, Fock build, read-back) is
                                one CUDA graph launch, captured on first use per kind of build; 0: eager
                                launches */
    double mixed_switch;     /* MIXED: coarse FP32-core macro-iterations until |dE| < mixed_switch */
    int32_t exact_engine;    /* J-engine of the FP64-accurate builds (every build in FEF_FP64, the
                                reference builds in FEF_MIXED): FEF_ENGINE_FP64 = native FP64 FMA,
                                FEF_ENGINE_DF64 = float-float arithmetic on the FP32 pipes (48-bit
                                significand, ~1e-14 relative; s/p Hermite classes, d-shell classes
                                stay FP64) */
    int32_t far_field;       /* 1: fragment pairs beyond cutoff_A (> 0) still interact, through the
                                multipoles (charge, dipole, second moments) of each fragment's nuclei and
                                electrons about its nuclear-charge centroid, y's potential Taylor-expanded
                                to second order about x's centroid (omega_x and the pair energies gain these
                                terms; the truncation error falls as R^-5); 0 (default): the plain cutoff */
    int32_t mixed_build;     /* what fef_build_fock computes in FEF_MIXED: FEF_MIXED_INCREMENT (default) =
                                J[D_ref] + J_fp32[D - D_ref] relative to the last FP64-accurate build (an
                                FP64 build when there is none); FEF_MIXED_WHOLE = the FP32-core J-engine
                                of the whole density, J_fp32[D] (FP64 accumulation, FP64 intra-fragment
                                G, V^y and energies), which becomes an inexact reference.  fef_iterate
                                ignores it (its schedule is fixed, see precision). */
} fef_options;

/* Fill *opt with the defaults: FP64, no cutoff, schwarz 1e-12, e_tol 1e-8, micro_e_tol 1e-11,
 * micro_comm_tol 1e-9, max_macro 100, max_micro 200, diis_size 8, superposition start,
 * mixed_switch 1e-6, use_graph 1, exact_engine FEF_ENGINE_FP64, far_field 0, mixed_build
 * FEF_MIXED_INCREMENT. */
void fef_default_options(fef_options* opt);

/* Build a context: validate and copy the inputs, then on the device normalise the basis, build
 * the Boys table, the one-electron matrices h^x = T^x + V^x(own nuclei) and S^x, the canonical
 * orthogonaliser X^x = U s^{-1/2} (s >= 1e-7), shell-pair Schwarz factors, the intra-fragment
 * two-electron tensor, the fragment-pair neighbour list within the cutoff, the environment nuclear
 * attraction sum_{y in N(x)} V^y (h~, the equation after Eq. wc) and the J-engine work lists.
 * cuda_stream: a cudaStream_t (NULL = default stream); it must outlive the context.  On success *out
 * owns device memory until fef_destroy, taken in stream order on cuda_stream from one memory pool per
 * device that the library shares between its contexts and that keeps up to 4 GiB cached after they
 * are destroyed (so that contexts of similar size are created again without cudaMalloc).  Errors: ARG (NULL pointers, an empty geometry or basis, an option out of range: diis_size
 * outside 1..8, NaN cutoff_A, non-positive or non-finite e_tol / micro tolerances, negative schwarz
 * or mixed_switch), BASIS, GEOM, CUDA.  Argument and option checks come before any device call. */
fef_status fef_create(const fef_geometry* geom, const fef_basis* basis, const fef_options* opt,
                      void* cuda_stream, fef_ctx** out);

/* n_ao_per_frag[n_frag] (may be NULL) and offsets[n_frag+1] (may be NULL): packed-block offsets in
 * doubles, offsets[x] = sum_{y<x} n_y^2.  Also usable to size every packed buffer. */
fef_status fef_ao_layout(const fef_ctx* ctx, int32_t* n_ao_per_frag, int64_t* offsets);

/* One FEF Fock build (Theory, "Fragment Mean Field", F~ with omega_x of Eq. wc / Eq. dp2e):
 *   F^x = h^x + G[D^x] + sum_{y in N(x)} (V^y + J[D^y])   for every fragment x.
 * D: packed densities to build from (becomes the context's current density), or NULL to use the
 * current densities.  F_out: packed output, or NULL.  on_device: 1 if D/F_out are device pointers.
 * The inter-fragment J is the fused McMurchie-Davidson J-engine: no ERI tensor is formed.  With
 * opt.far_field, omega_x also holds the multipole field of the fragments beyond the cutoff.
 * FP64 mode: the full FP64 J-engine.  MIXED with opt.mixed_build = FEF_MIXED_INCREMENT:
 * J[D^y] = J[D_ref] + J_fp32[D^y - D_ref] relative to the last FP64 build of this context; without
 * one the build is FP64 and becomes the reference.  MIXED with FEF_MIXED_WHOLE: J_fp32[D^y], the
 * FP32-core J-engine of the whole density (its error against the FP64 build is what the FP32 core
 * alone costs).  Errors: ARG, CUDA, NUMERIC. */
fef_status fef_build_fock(fef_ctx* ctx, const double* D, double* F_out, int on_device);

/* FEF self-consistency (Theory, "Fragment Mean Field": omega_x relaxed to self-consistency).
 * Start from the option's start densities (superposition of isolated-fragment RHF densities, the
 * learned warm start (fef_set_warm_start), or the current/given ones); each macro-iteration k builds omega^(k) from
 * D^(k-1) of all fragments and solves every fragment's RHF in its frozen field (DIIS, canonical
 * orthogonalisation, aufbau) to get D^(k); stops when |dE_tot| and max_x |dE_x| < e_tol.
 * n_macro_out (nullable): macro-iterations done; final_dE_out (nullable): last |dE_tot|.
 * Errors: NOT_CONVERGED (context stays valid, densities are the last iterate), NUMERIC, CUDA. */
fef_status fef_iterate(fef_ctx* ctx, int32_t* n_macro_out, double* final_dE_out);

/* The non-interacting mean field (Theory, "Fragment Mean Field", the first of the two mean-field
 * choices: F = h(1) + (2J - K) per fragment, inter-fragment terms left to perturbation theory).
 * Solves every fragment's RHF without environment field (core guess, DIIS) and makes these
 * densities the current ones, so that fef_energies then gives the energies of the unperturbed
 * product state (E_x^int + half the first-order pair terms) and fef_build_fock(ctx, NULL, ...)
 * the Fock matrices with omega_x built from the unperturbed densities of the other fragments.
 * These are also the superposition start of fef_iterate.
 * Errors: NOT_CONVERGED (a fragment RHF; densities are the last iterate), NUMERIC, CUDA. */
fef_status fef_noninteracting_scf(fef_ctx* ctx);

/* Reference energies of the current densities (from <H_x> and <H_xy> of the Hamiltonian partition,
 * Eqs. NHx, NHxy, clusterH, pairs counted once):
 *   E_int[x] = tr[D^x (2 h^x + G[D^x])]/2 + sum_{A<B in x} Z_A Z_B / R_AB
 *   E_xy     = tr[D^x V^y] + tr[D^y V^x] + tr[D^x J[D^y]] + sum_{A in x, B in y} Z_A Z_B / R_AB
 *   E_total  = sum_x E_int[x] + sum_{x<y in N} E_xy;   E_frag[x] = E_int[x] + (1/2) sum_y E_xy.
 * With opt.far_field the pairs beyond the cutoff add their multipole interaction energies to E_total
 * and half to each E_frag.  Any output pointer may be NULL; E_frag/E_int are [n_frag] host arrays. */
fef_status fef_energies(fef_ctx* ctx, double* E_frag, double* E_total, double* E_int);

/* Monomer second-order energy of the FEF cluster perturbation theory (Eq. EM2, with the first-order
 * monomer doubles of Eq. monDoubles): with each fragment's canonical FEF orbitals (F^x C = S^x C eps
 * of the current densities' Fock matrices, canonical orthogonalisation, aufbau) the zeroth-order
 * monomer effective Hamiltonian is the diagonal Fock operator and the doubles are driven by the
 * fragment's own two-electron interaction (the environment field is one-body), so
 *   E_M2^x = sum_{ij occ, ab virt} (ia|jb) [2 (ia|jb) - (ib|ja)] / (eps_i + eps_j - eps_a - eps_b).
 * E_m2[n_frag] (host, nullable) per fragment, *E_m2_total (nullable) their sum.  The fragments'
 * integrals are recomputed into temporary device memory for the call (n^2 (n+1)^2 / 4 doubles per
 * fragment of n AOs).  Errors: ARG (no densities), CUDA. */
fef_status fef_energy_m2(fef_ctx* ctx, double* E_m2, double* E_m2_total);

/* Dimer second-order energy of the FEF cluster perturbation theory (Eq. ED2, with the first-order
 * dimer doubles of Eq. dimDoubles), summed over the fragment pairs within the cutoff (each pair
 * once): with the canonical FEF orbitals of both fragments the dimer doubles excite one electron on
 * each fragment and interact directly only (no inter-fragment exchange in the product ansatz):
 *   E_D2^{xy} = 4 sum_{i,a in x; j,b in y} (ia|jb)^2 / (eps_i + eps_j - eps_a - eps_b).
 * E_d2_frag[n_frag] (host, nullable) = half of each fragment's pair terms, *E_d2_total (nullable) =
 * sum over pairs.  Fragments of s and p shells: the integrals come from the Hermite transition
 * densities of the occupied-virtual pairs (no AO integral block); with d shells the pair integral
 * blocks are computed into temporary device memory.  Both in chunks of pairs.
 * Errors: ARG (no densities), CUDA. */
fef_status fef_energy_d2(fef_ctx* ctx, double* E_d2_frag, double* E_d2_total);

/* Checkpoint / resume: copy the current packed densities out, or replace them. */
fef_status fef_get_densities(const fef_ctx* ctx, double* D_out, int on_device);
fef_status fef_set_densities(fef_ctx* ctx, const double* D_in, int on_device);

/* Counters of the last Fock build / iteration.  Any pointer may be NULL.
 *   shell_quartets: inter-fragment shell quartets (a<=b in x, c<=d in y, x<y) surviving the cutoff
 *                   and Schwarz screening, counted once per build;
 *   prim_quartets:  primitive quartets evaluated per build;
 *   n_pairs:        fragment pairs in the neighbour list;
 *   jengine_ms:     device time of the J-engine launches of the last fef_build_fock, or summed over
 *                   the builds of the last fef_iterate (CUDA events on the context stream);
 *   kernel_launches: kernels launched by this library (all contexts) since it was loaded;
 *   class_quartets: [25] primitive quartets of the surviving shell quartets per Hermite class,
 *                   index L_bra*5 + L_ket with L = l_a + l_b of the shell pair.
 * ctx may be NULL when only kernel_launches is asked for. */
fef_status fef_stats(const fef_ctx* ctx, int64_t* shell_quartets, int64_t* prim_quartets, int64_t* n_pairs,
                     double* jengine_ms, int64_t* kernel_launches, int64_t* class_quartets);

/* Per-macro-iteration log of the last fef_iterate (record 0 = the start densities).  Each record is
 * 9 doubles: k, E_total, |dE_total|, max_x |dE_x|, max micro-iterations over fragments, summed
 * micro-iterations, J-engine ms of the Fock build, fragment-SCF ms (CUDA events), and 1.0 if the
 * build used the FP32 core (MIXED) else 0.0.  Copies min(n, max_records) records into records
 * (host, nullable); *n_records (nullable) gets n. */
fef_status fef_history(const fef_ctx* ctx, int32_t max_records, double* records, int32_t* n_records);

/* Per-fragment state of the last fragment-RHF launch (the start SCF, or the last macro-iteration's):
 * micro_iters[n_frag] = micro-iterations to convergence, or -max_micro when the fragment did not
 * converge; homo_lumo_gap[n_frag] = lowest virtual minus highest occupied orbital energy of the last
 * Roothaan step (hartree; aufbau is ill-defined when it is near 0); E_scf[n_frag] = tr[D (h + omega +
 * F)]/2 + own nuclear repulsion.  Host arrays, each nullable.  Errors: ARG, CUDA. */
fef_status fef_fragment_status(const fef_ctx* ctx, int32_t* micro_iters, double* homo_lumo_gap, double* E_scf);

/* Message of the last failing call on ctx, or, when ctx is NULL, of the last failed context-free call
 * (fef_create, fef_fragment_rhf_noalloc, fef_measure_fma_peak) made by the calling host thread (the
 * context-free message is thread-local; the pointer stays valid until that thread's next failing
 * context-free call). */
const char* fef_last_error(const fef_ctx* ctx);

/* Free the context and all its device memory (waits for the device, then returns the memory to the
 * library's pool).  NULL is a no-op. */
void fef_destroy(fef_ctx* ctx);

/* ---------------------------------------------------------------------------------------------
 * Tile plans of the inter-fragment J-engine.  The plan decides only how the work of a Fock build is
 * cut into warp-sized items and scheduled; every plan computes the same J (Eq. dp2e) up to the
 * order of floating-point additions.  A work item is one warp's tile of 32 bra primitive pairs of
 * one fragment of a pair against a chunk of the partner's primitive pairs of one Hermite class.
 * ------------------------------------------------------------------------------------------- */
enum { FEF_JENGINE_FP64 = 0, FEF_JENGINE_FP32 = 1, FEF_JENGINE_DF64 = 2 };

typedef struct {
    int32_t persistent;     /* 1: one persistent kernel per register tier (Hermite integrals in registers,
                               in shared memory, float-float), whose warps take items from a queue sorted
                               by decreasing cost (all fragment pairs and classes in one launch); the
                               tiers run concurrently.  0: one launch per class pair over whole ket
                               ranges (ket_chunk unused).  2: the same class-pair kernels launched on
                               three streams (graph branches when captured), largest classes first,
                               so that they run concurrently; ket_chunk cuts the tiles of the register
                               classes into chunks (one warp each; the float-float and shared-memory
                               classes use whole ranges). */
    int32_t ket_chunk[25];  /* ket primitive pairs per item for the class pair L_bra*5 + L_ket
                               (L = l_a + l_b of the shell pair); 0 = the partner's whole class range */
    double tuned_ms;        /* J-engine time of one build measured by fef_autotune (0: not tuned) */
} fef_tile_plan;

/* Read or replace the plan of one engine (FEF_JENGINE_FP64: FP64 builds; FEF_JENGINE_FP32: the FP32-core
 * builds of FEF_MIXED; FEF_JENGINE_DF64: float-float builds).  Default plans: persistent (1) for
 * FEF_JENGINE_FP64 and concurrent class-pair launches (2) for the other two; whole ket ranges, except that
 * an s/p or register d class whose whole-range work items would give fewer than 32 warps per SM (small
 * workloads) is cut into 64-pair ket chunks in the FP64 and FP32 plans.  Setting rebuilds the work queues
 * (synchronous).  Errors: ARG, CUDA. */
fef_status fef_get_tile_plan(const fef_ctx* ctx, int32_t engine, fef_tile_plan* out);
fef_status fef_set_tile_plan(fef_ctx* ctx, int32_t engine, const fef_tile_plan* plan);

/* Autotuner: times candidate plans of one engine on this context's own workload with CUDA events, each
 * pass captured once into a CUDA graph and replayed (fef_iterate runs its builds as graph launches),
 * and installs the fastest.  It chooses the ket chunk of each class pair (from whole range, 1024, 256, 64
 * ket pairs; classes in decreasing order of cost) on every k-th fragment pair, k chosen so that one
 * timed pass takes about budget_ms/64, then, when a full build fits the budget, persistent queues
 * against one launch per class pair, serial or concurrent, and against the plan in place when the
 * call began (kept unless a tuned plan is faster).  Each candidate is timed reps times (best kept) after a warm-up.
 * The timed passes run on the context's current densities, prepared as a build of that engine prepares
 * them (Hermite densities; for FEF_JENGINE_FP32 the FP32 records relative to the stored reference
 * density, or to zero before the first reference build).  Runs between builds (it overwrites the
 * J-engine accumulators and the per-build Hermite data; the next build recomputes both from its own
 * density; the reference of FEF_MIXED is left unchanged).  out (nullable) receives the chosen plan.
 * Errors: ARG, CUDA. */
fef_status fef_autotune(fef_ctx* ctx, int32_t engine, int32_t reps, double budget_ms, fef_tile_plan* out);

/* Measure this GPU's FP64 and FP32 FMA throughput with a register-resident FMA chain kernel.
 * Outputs (nullable) in FLOP/s, counting one FMA as 2 FLOP.  Errors: CUDA. */
fef_status fef_measure_fma_peak(double* fp64_flops, double* fp32_flops, double* sm_clock_mhz);

/* ---------------------------------------------------------------------------------------------
 * Learned warm start.  The paper has no learned component: this is an accelerator of the FEF
 * iterations that leaves the fixed point unchanged (the plain FEF loop still converges the result
 * and judges the energy).  A small perceptron maps the environment of each fragment to the change
 * of its density from the isolated-fragment RHF density, in the fragment's molecule-fixed frame
 * (axes from atoms 0, 1, 2 in input order).  It needs fragments of one kind (same atoms, s/p basis).
 * ------------------------------------------------------------------------------------------- */
typedef struct fef_mlp fef_mlp;

/* Network Y = W3 tanh(W2 tanh(W1 X + b1) + b2) + b3 with n_in inputs, two hidden layers of n_hidden,
 * n_out outputs; FP32 weights, Glorot-uniform initialisation from seed (splitmix64).  All work on
 * cuda_stream.  Errors: ARG, CUDA. */
fef_status fef_mlp_create(int32_t n_in, int32_t n_hidden, int32_t n_out, uint64_t seed, void* cuda_stream,
                          fef_mlp** out);
void fef_mlp_destroy(fef_mlp* m);
/* Get (set = 0) or set (set = 1) the flat parameters W1 (n_in x n_hidden, row-major), b1, W2, b2, W3, b3
 * through the HOST array params (nullable); *n_params (nullable) gets their number.  Setting resets Adam. */
fef_status fef_mlp_params(fef_mlp* m, float* params, int64_t* n_params, int32_t set);
/* Affine scaling used by fef_mlp_predict and by the warm start: the network sees (X - in_shift)/in_scale
 * and its output y becomes out_shift + out_scale * y.  Host arrays of n_in / n_out floats. */
fef_status fef_mlp_set_scaling(fef_mlp* m, const float* in_shift, const float* in_scale, const float* out_shift,
                               const float* out_scale);
/* Mean squared error L = sum (Y - T)^2 / (n n_out) of the raw network (no scaling) on DEVICE arrays
 * X [n x n_in], T [n x n_out], and its gradient into the DEVICE array grad [n_params] (nullable). */
fef_status fef_mlp_loss_grad(fef_mlp* m, const float* X, const float* T, int32_t n, float* loss, float* grad);
/* Adam (beta 0.9/0.999, eps 1e-8) on mini-batches of the raw network, shuffled every epoch; DEVICE
 * X, T as above; *final_loss (nullable) = mean squared error over the last epoch. */
fef_status fef_mlp_train(fef_mlp* m, const float* X, const float* T, int32_t n, int32_t epochs, int32_t batch,
                         float lr, float* final_loss);
/* Y [n x n_out] = scaled network(X [n x n_in]); DEVICE arrays. */
fef_status fef_mlp_predict(fef_mlp* m, const float* X, float* Y, int32_t n);
const char* fef_mlp_last_error(const fef_mlp* m);

/* Features of the learned warm start for the densities D (packed, becomes the current density; NULL =
 * current): X [n_frag x n_feat] = per atom the potential and field (frame components) of all neighbour
 * fragments' nuclei and electrons (4 n_atoms values), then the multipole estimate of the environment
 * operator: -(phi S + grad phi . <r> + (1/2) hess phi : <r r>) with phi the potential of the
 * neighbours' charges, dipoles and second moments (about their nuclear-charge centroids) expanded to
 * second order about x's centroid, in the Loewdin basis (S^{-1/2} omega S^{-1/2}) and the
 * molecule-fixed frame, upper triangle (n_pack values): n_feat = 4 n_atoms + n_pack.  No Fock build.  Y_local [n_frag x n_pack] = the
 * density in the Loewdin basis (S^{1/2} D S^{1/2}, S^{1/2} symmetric) expressed in the molecule-fixed
 * frame, upper triangle row-major (n_pack = n(n+1)/2).  X, Y_local are
 * host arrays, or device arrays when on_device = 1; either may be NULL.  *n_feat, *n_pack (nullable)
 * are 0 when the fragments are not of one kind.  Errors: ARG, CUDA. */
fef_status fef_learned_features(fef_ctx* ctx, const double* D, float* X, float* Y_local, int on_device,
                                int32_t* n_feat, int32_t* n_pack);
/* Attach the network used by fef_iterate when opt.start = FEF_START_LEARNED (NULL detaches; the
 * caller keeps ownership).  Its outputs are the change of the local-frame Loewdin-basis density from
 * the isolated-fragment one; the start is D_isolated + S^{-1/2} (that change, rotated back) S^{-1/2}. */
fef_status fef_set_warm_start(fef_ctx* ctx, fef_mlp* m);

/* Batched closed-shell RHF of independent fragments in frozen fields, for callers that cannot
 * allocate device memory.  The paper has no counterpart: this is a service entry point of this
 * library.  Some callers own every byte of device memory themselves (a dynamics or embedding
 * driver that runs under a fixed device-memory budget or hands out memory from its own pool), or
 * must not pay for, or serialise on, cudaMalloc/cudaFree inside a time step; this call allocates
 * nothing.
 *
 * It runs the same kernels as the fragment RHF of fef_iterate (canonical orthogonaliser
 * X = U s^{-1/2} dropping s < 1e-7, then the device micro loop: F = h + omega + C D, Pulay DIIS,
 * cyclic Jacobi, aufbau, D = 2 C_occ C_occ^T until |dE| < micro_e_tol and max|FDS-SDF| <
 * micro_comm_tol).  Its working memory (orthogonalisers, DIIS history, offsets, status flag) lives
 * in a fixed 16 MiB device array inside libfef.so, held by every GPU that loads the library until
 * the process exits.
 *   n_frag              1..65535 fragments, batched in one launch.
 *   n_ao, n_occ, e_nn   HOST arrays [n_frag]: AOs (1..56), doubly occupied orbitals, nuclear
 *                       repulsion of the fragment's own nuclei (hartree).
 *   S, h, omega         DEVICE packed n_x*n_x blocks (overlap, core Hamiltonian, environment field;
 *                       omega may be NULL for isolated fragments).
 *   eri_c               DEVICE, per fragment the full n_x^4 tensor
 *                       C[mu nu][lambda sigma] = (mu nu|lambda sigma) - (mu lambda|nu sigma)/2,
 *                       blocks concatenated.
 *   D_start             DEVICE packed start densities, or NULL for the core guess (F = h + omega).
 *   D_out, F_out        DEVICE packed outputs: converged densities and their Fock matrices.
 *   E_scf               DEVICE [n_frag] output: tr[D(h + omega + F)]/2 + e_nn.
 *   opt                 micro_e_tol, micro_comm_tol, max_micro, diis_size are used (NULL: defaults).
 *   cuda_stream         stream for all work; the call reads the fragments' status back and
 *                       synchronises the stream before returning.
 * Limits: the batch must fit the 16 MiB scratch: per fragment n_x^2 doubles of orthogonaliser and
 * 2*diis_size*max_n^2 doubles of DIIS history (about 700 13-AO fragments with diis_size 8), else
 * FEF_ERR_ARG, checked on the host before any device work.  Set-up: the first call on each device,
 * with that device current, resolves the scratch's device address with cudaGetSymbolAddress and
 * caches it; make that first call before any stream capture begins.  All calls share the scratch
 * and it keeps the last call's contents (the call clears what must start at zero): calls whose
 * device work overlaps (two streams, two host threads) race on it.  Errors (message from
 * fef_last_error(NULL) on the calling thread): ARG (also when a device bounds check fails), CUDA,
 * NOT_CONVERGED (outputs hold the last iterate), NUMERIC. */
fef_status fef_fragment_rhf_noalloc(int32_t n_frag, const int32_t* n_ao, const int32_t* n_occ, const double* e_nn,
                                    const double* S, const double* h, const double* omega, const double* eri_c,
                                    const double* D_start, double* D_out, double* F_out, double* E_scf,
                                    const fef_options* opt, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* FEF_H */
