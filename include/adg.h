/*
 * adg.h -- C ABI of libadg.so, a GB300 (sm_103a) implementation of the hot
 * path of AutoDock-GPU-style protein-ligand docking (arXiv 2007.03678).
 *
 * The paper's statement of the problem (Sec. 1, 1.1, 2.2): one receptor given
 * as interaction grid maps (atom-type affinity, electrostatic and
 * desolvation maps, Sec. 2.2.1 and 2.3), many ligands given as atom
 * coordinates, types, charges and rotatable bonds, and the run parameters
 * nrun / nev (Sec. 1.1); out come the best pose and energy of each of the
 * nrun independent Lamarckian-GA runs (Sec. 1, 1.1).  The receptor maps are
 * uploaded once and stay resident, and the context keeps its device memory
 * for reuse between ligands (Sec. 2.2.3).
 *
 * Conventions for every call:
 *  - Return value: ADG_OK (0) or a negative ADG_E* code; adg_strerror() gives
 *    its text.  On error nothing is written to the caller's outputs except
 *    where stated, and no exception crosses the ABI.
 *  - Ownership: the caller owns every pointer it passes; the library copies
 *    what it needs.  Handles are freed only by their *_destroy call; a
 *    receptor or ligand may be destroyed after the context that made it.
 *  - "device" pointers are CUDA global-memory addresses on the context's
 *    device (for example a torch tensor's data_ptr()); "host" pointers are
 *    ordinary CPU memory.  Device work is ordered on the context's stream.
 *  - Threading: one context per host thread.
 *  - Units: Angstrom, radian, kcal/mol.  Floating point is IEEE binary32.
 */
#ifndef ADG_H
#define ADG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ADG_NTYPES 7          /* ligand atom types C, A, N, NA, OA, HD, S (map index 0..6) */
#define ADG_NMAPS 9           /* 7 type maps, 7 = electrostatic, 8 = desolvation           */
#define ADG_MAP_ELEC 7
#define ADG_MAP_DESOLV 8
#define ADG_MAX_ATOMS 128
#define ADG_MAX_TORS 16
#define ADG_MAX_GENES (7 + ADG_MAX_TORS)
#define ADG_TRACE_WIDTH 12    /* int32 words per offspring in adg_dock_trace.decisions */

enum {
    ADG_OK = 0,
    ADG_EINVAL = -1,   /* null pointer, negative or inconsistent size            */
    ADG_ETYPE = -2,    /* atom type outside 0..ADG_NTYPES-1                      */
    ADG_ETOOBIG = -3,  /* more than ADG_MAX_ATOMS atoms or ADG_MAX_TORS torsions */
    ADG_EGRID = -4,    /* fewer than 2 points on an axis or spacing <= 0         */
    ADG_ECUDA = -5,    /* a CUDA runtime call failed                             */
    ADG_ETIMEOUT = -6, /* a bounded device-side wait expired                     */
    ADG_ENOMEM = -7,   /* device or host allocation failed                       */
    ADG_ETOPO = -8     /* bonds do not form one tree, or a torsion is not a bond */
};

typedef struct adg_ctx adg_ctx;
typedef struct adg_receptor adg_receptor;
typedef struct adg_ligand adg_ligand;

/* Force-field table (AutoDock4 free-energy model, paper Sec. 1: vdW,
 * H-bond, electrostatics with a distance-dependent dielectric, desolvation,
 * torsional entropy).  Per-type arrays are indexed by map index 0..6.
 *   pair vdW/H-bond: generalised n-m potential with minimum -eps at r0;
 *     12-6 with r0 = (Rii_i+Rii_j)/2, eps = sqrt(epsii_i epsii_j), weight w_vdw;
 *     12-10 between a donor and an acceptor with the acceptor's hb_R/hb_eps,
 *     weight w_hb; value capped at e_cap.
 *   elec: w_elec * coulomb * q_i q_j / (eps(r) r), Mehler-Solmajer
 *     eps(r) = ms_A + B / (1 + ms_k exp(-ms_lambda B r)), B = ms_eps0 - ms_A.
 *   desolvation: w_desolv [(solpar_i + qasp|q_i|) vol_j + (solpar_j + qasp|q_j|) vol_i]
 *     * exp(-r^2 / (2 sigma^2)).
 *   r is floored at r_min.  Maps use a smooth cutoff switching from 1 at
 *   map_r_on to 0 at map_r_off.  Outside the grid box an atom pays k_out d^2. */
typedef struct {
    float Rii[ADG_NTYPES], epsii[ADG_NTYPES], vol[ADG_NTYPES], solpar[ADG_NTYPES];
    int32_t hb_donor[ADG_NTYPES], hb_acceptor[ADG_NTYPES];
    float hb_R[ADG_NTYPES], hb_eps[ADG_NTYPES];
    float w_vdw, w_hb, w_elec, w_desolv, w_tors;
    float qasp, sigma, coulomb;
    float ms_A, ms_eps0, ms_lambda, ms_k;
    float r_min, e_cap, map_r_on, map_r_off, k_out;
} adg_forcefield;

/* Grid: n[0..2] points along x, y, z; node (i,j,k) at origin + (i,j,k)*spacing.
 * Map storage is [map][z][y][x] (x fastest), ADG_NMAPS maps. */
typedef struct {
    int32_t n[3];
    float origin[3];
    float spacing;
} adg_grid_desc;

/* Ligand description (host memory).  xyz[3*natoms] is the reference
 * conformation; type[natoms] map indices; charge[natoms]; bonds[2*nbonds]
 * must form one tree (the library builds the torsion tree from it);
 * tors[2*ntors] lists rotatable bonds (either orientation: the side not
 * holding `root` is the one that moves). */
typedef struct {
    int32_t natoms;
    const float* xyz;
    const int32_t* type;
    const float* charge;
    int32_t nbonds;
    const int32_t* bonds;
    int32_t ntors;
    const int32_t* tors;
    int32_t root;
} adg_ligand_desc;

enum { ADG_LS_NONE = 0, ADG_LS_SOLIS_WETS = 1, ADG_LS_ADADELTA = 2 };

/* Search parameters.  nrun and nev follow the paper (Sec. 1.1): nrun
 * independent LGA runs per ligand, each stopping once it has spent nev
 * energy evaluations (checked between generations, so the last generation
 * may overshoot).  One energy call or one energy+gradient call is one
 * evaluation.  The remaining defaults are readings of "other parameters
 * default" (Sec. 2.3); adg_search_params_default() fills them in. */
typedef struct {
    int32_t nrun, pop_size, nev, max_gen, ls_method, ls_max_iters, elitism;
    float ls_rate, crossover_rate, mutation_rate, tournament_rate;
    float sw_rho0, sw_rho_min, sw_expand, sw_contract;
    int32_t sw_succ, sw_fail;
    float sw_scale_t, sw_scale_rot, sw_scale_tors;
    float ad_rho, ad_eps;
    float mut_t, mut_rot, mut_tors;
    uint64_t seed;      /* Philox key                                          */
    uint32_t lig_id;    /* Philox counter word 0 of the first ligand in a call */
    int32_t autostop;   /* nonzero: stop a run early (paper Sec. 1.1)          */
    float stopstd;      /* ... once the standard deviation of its best energy over the last 10
                           generations is below stopstd (kcal/mol)            */
    int32_t pad0;
} adg_search_params;

/* Result of one run (host memory).  genes: [t(3), q(4) (w,x,y,z), theta(T)];
 * xyz: posed coordinates of the best genotype, 3*natoms floats. */
typedef struct {
    float best_energy;
    int32_t generations;
    int64_t evals;
    float genes[ADG_MAX_GENES];
    float xyz[3 * ADG_MAX_ATOMS];
} adg_result;

/* Optional record of the first `ngen` generations of a one-ligand dock, for
 * replaying the GA decisions.  All arrays are host memory, caller-allocated:
 *   decisions [nrun][ngen][pop][12] int32: parent1, parent2, crossover lo,
 *             crossover hi (-1 when no crossover), mutation block mask,
 *             local search applied, tournament candidates a1, b1, a2, b2
 *             (-1 for the elite slot), 0, 0
 *   genes     [nrun][ngen][pop][7+T] population after each generation
 *   energies  [nrun][ngen][pop]
 *   init_genes[nrun][pop][7+T] and init_energies[nrun][pop]: generation 0.
 * Any pointer may be NULL to skip that array. */
typedef struct {
    int32_t ngen;
    int32_t* decisions;
    float* genes;
    float* energies;
    float* init_genes;
    float* init_energies;
} adg_dock_trace;

/* Error code -> static text.  Never fails. */
const char* adg_strerror(int code);

/* Defaults: pop 150, nev 2,500,000, max_gen 27,000, Solis-Wets, 300
 * iterations, elitism 1, ls_rate 1, crossover 0.8, mutation 0.02,
 * tournament 0.6, rho0 1, rho_min 0.01, x2 after 4 successes, x0.5 after 4
 * failures, step scales 1 A / 0.5 rad / 0.5 rad, ADADELTA rho 0.8 eps 0.01,
 * mutation half-widths 2 A / pi/2 / pi/2, seed 42, nrun 10, autostop off,
 * stopstd 0.15 kcal/mol. */
void adg_search_params_default(adg_search_params* p);

/* Context: selects `device`, creates or adopts a CUDA stream (`stream` may be
 * NULL for a library-owned stream, else a cudaStream_t the caller keeps
 * alive), and owns a reusable device arena (context and memory reuse,
 * paper Sec. 2.2.3).  *out receives the handle. */
int adg_ctx_create(adg_ctx** out, int device, void* stream);
int adg_ctx_destroy(adg_ctx* ctx);
/* Block until the context's stream has drained; reports a deferred CUDA error. */
int adg_sync(adg_ctx* ctx);
/* Detail text of the last ADG_ECUDA on this context ("" if none). */
const char* adg_ctx_last_error(const adg_ctx* ctx);

/* Receptor grid maps from receptor atoms (the role AutoGrid4 plays in the
 * paper, Sec. 2.3): for every node p
 *   M_t(p) = min(e_cap, sum_j S(r)[vdW/HB(t, type_j)(r) + w_desolv (solpar_t vol_j
 *            + (solpar_j + qasp|q_j|) vol_t) G(r)]),        t = 0..6
 *   M_e(p) = sum_j S(r) w_elec coulomb q_j / (eps(r) r)
 *   M_d(p) = sum_j S(r) w_desolv qasp vol_j G(r)
 * with S the smooth cutoff and G(r) = exp(-r^2/(2 sigma^2)).
 * rec_xyz[3*nrec], rec_type[nrec], rec_q[nrec]: host.  maps_out: device,
 * ADG_NMAPS*nz*ny*nx floats, [map][z][y][x].  Asynchronous on the stream. */
int adg_maps_build(adg_ctx* ctx, const adg_forcefield* ff, const adg_grid_desc* grid, int nrec,
                   const float* rec_xyz, const int32_t* rec_type, const float* rec_q, float* maps_out);

/* Resident receptor (paper Sec. 2.2.3: grids sent once and left on device).
 * maps: ADG_NMAPS*nz*ny*nx floats [map][z][y][x], host memory when
 * maps_on_device == 0, else device memory.  The library keeps its own
 * packed copy; the caller may free `maps` once this returns. */
int adg_receptor_create(adg_ctx* ctx, const adg_grid_desc* grid, const float* maps, int maps_on_device,
                        adg_receptor** out);
int adg_receptor_destroy(adg_receptor* rec);

/* Ligand: copies the description, builds the torsion tree (rigid fragments,
 * moving set of each rotatable bond, deepest-first application order) and
 * the intramolecular pair list (pairs in different rigid fragments and more
 * than 3 bonds apart), with per-pair coefficients from `ff`, and uploads it. */
int adg_ligand_create(adg_ctx* ctx, const adg_forcefield* ff, const adg_ligand_desc* desc, adg_ligand** out);
int adg_ligand_destroy(adg_ligand* lig);
/* Sizes of a built ligand: atoms, torsions, intramolecular pairs, the sum
 * over torsions of the moving-set sizes, and the bytes uploaded for it. */
typedef struct {
    int32_t natoms, ntors, npairs, sum_moving;
    int64_t device_bytes;
} adg_ligand_stats;
int adg_ligand_info(const adg_ligand* lig, adg_ligand_stats* out);

/* Fixed-length description of a ligand, the input of the triage network
 * (adg_mlp_*); no counterpart in the paper.  out: host [ADG_NDESC] floats =
 * atoms, torsions, intramolecular pairs, atom counts of the 7 types (C, A, N,
 * NA, OA, HD, S), sum |q|, sum q^2, radius of gyration and largest distance
 * from the centroid of the input conformation (A), rigid fragments, mean
 * moving-set size per torsion. */
#define ADG_NDESC 16
int adg_ligand_descriptors(const adg_ligand* lig, float* out);

/* Random-stream identity of a ligand.  Every Philox counter of a dock call
 * carries a ligand word: by default p->lig_id + the ligand's index in the
 * call; after adg_ligand_set_stream_id(lig, id) with 0 <= id < 2^32, `id`
 * in every call (so a ligand docked alone, in any batch or in any subset of
 * a batch gives the same runs); id = -1 restores the default. */
int adg_ligand_set_stream_id(adg_ligand* lig, int64_t id);

enum { ADG_GRAD_NONE = 0, ADG_GRAD_GENES = 1, ADG_GRAD_TANGENT = 2 };

/* Energy (and gradient) of npose genotypes of one ligand (Sec. 1: the
 * AD4 energy evaluated on LGA genotypes).  Genotype = [t(3), q(4) (w,x,y,z)
 * used as q/|q|, theta(T) as deltas from the input conformation].  The pose
 * applies the torsions deepest first about their reference axes, then
 * x' = R(q/|q|)(x - centroid) + t.  Energy = intermolecular (trilinear map
 * interpolation + out-of-box restraint) + intramolecular pair terms.
 *   genes:  device [npose][7+T]
 *   energy: device [npose]
 *   grad:   device; NULL when grad_kind == ADG_GRAD_NONE;
 *           ADG_GRAD_GENES   -> [npose][7+T]: dE/dt, dE/dq, dE/dtheta
 *           ADG_GRAD_TANGENT -> [npose][6+T]: dE/dt, torque, dE/dtheta
 * Asynchronous on the context's stream. */
int adg_score(adg_ctx* ctx, const adg_receptor* rec, const adg_ligand* lig, const float* genes, int npose,
              float* energy, float* grad, int grad_kind);

/* adg_score over the poses of several ligands in one launch per
 * atoms-per-lane width (the ligands of a differentiable batch).  Ligand i
 * owns npose[i] consecutive rows, in ligand order (host array [nlig]); every
 * row is ADG_MAX_GENES floats:
 *   genes:  device [total][ADG_MAX_GENES]; a row holds its ligand's 7+T genes
 *           in front, the rest is ignored
 *   energy: device [total]
 *   grad:   device [total][ADG_MAX_GENES], NULL when grad_kind ==
 *           ADG_GRAD_NONE; a row gets 7+T (ADG_GRAD_GENES) or 6+T
 *           (ADG_GRAD_TANGENT) values in front and zeros after them
 * Each pose gets the same values as adg_score gives it.  The widths run on
 * concurrent streams that fork from and join back into the context's stream.
 * The launch tables (which block serves which ligand's rows) live in a device
 * buffer the context keeps and re-uploads, in stream order, only when a call's
 * tables differ from the previous call's.  ADG_EINVAL on a null argument, a
 * negative count or a ligand of another context, ADG_ETOOBIG beyond 2^30 rows;
 * asynchronous on the context's stream. */
int adg_score_multi(adg_ctx* ctx, const adg_receptor* rec, const adg_ligand* const* ligs, int nlig, const int* npose,
                    const float* genes, float* energy, float* grad, int grad_kind);

/* Posed coordinates of npose genotypes: xyz device [npose][natoms][3]. */
int adg_pose(adg_ctx* ctx, const adg_ligand* lig, const float* genes, int npose, float* xyz);

/* Dock nlig ligands against one receptor: p->nrun independent Lamarckian GA
 * runs each (Sec. 1, 1.1), every run a population of p->pop_size genotypes
 * refined by Solis-Wets or ADADELTA local search, until p->nev evaluations
 * or p->max_gen generations.  out: host, caller-allocated [nlig][p->nrun].
 * trace: NULL, or (nlig == 1 only) the record described at adg_dock_trace.
 * Returns when the results are in `out`. */
int adg_dock(adg_ctx* ctx, const adg_receptor* rec, const adg_ligand* const* ligs, int nlig,
             const adg_search_params* p, adg_result* out, adg_dock_trace* trace);

/* adg_dock that also reports each run's best-energy trace: best_trace, host,
 * caller-allocated [nlig][p->nrun][ntrace]; entry k is the lowest energy of
 * the run's population after generation k+1 (with elitism, the best energy
 * found so far).  Entries past the run's last generation repeat its final
 * best energy.  The early part of this trace (the mechanism behind the
 * paper's autostop, Sec. 1.1) feeds the triage network. */
int adg_dock_traced(adg_ctx* ctx, const adg_receptor* rec, const adg_ligand* const* ligs, int nlig,
                    const adg_search_params* p, adg_result* out, float* best_trace, int ntrace);

/* Launch accounting of a context, for measurement.  Counts every kernel the
 * library launched on the context since the last reset; when timing is on
 * (adg_ctx_set_timing), the generation loops of each adg_dock call are
 * bracketed by CUDA events: gen_kernel_ms adds the span from the first
 * group's loop start to the last group's loop end (the groups of a call run
 * concurrently), gen_timed the generations of its longest group, so
 * gen_kernel_ms / gen_timed is the time of one generation of all its runs. */
typedef struct {
    int64_t kernel_launches;  /* all kernels launched by the library       */
    int64_t gen_launches;     /* generation kernels (selection + LS) only  */
    double gen_kernel_ms;     /* event-timed span of the generation loops  */
    int64_t gen_timed;        /* generation rounds in that span            */
    int64_t h2d_bytes;        /* host -> device bytes copied by the library */
    int64_t d2h_bytes;        /* device -> host bytes copied by the library */
    int64_t dock_groups;      /* ligand groups (one graph each) of adg_dock */
    int64_t tune_launches;    /* kernels launched to tune launch geometry   */
} adg_stats;

int adg_ctx_set_timing(adg_ctx* ctx, int enable);
/* Copy the counters to *out; zero them when reset != 0.  (adg_dock reads
 * its timing events before it returns, so this does not wait.) */
int adg_ctx_stats(adg_ctx* ctx, adg_stats* out, int reset);

/* How adg_dock drives its generation loop (no counterpart in the paper).
 * enable != 0 (default): one CUDA graph per ligand group -- initial
 * population, a device-side WHILE loop of (generation, bookkeeping, loop
 * control) that runs until no run of the group is active, final poses -- so
 * the host launches once per group.  enable == 0: the same kernels launched
 * from the host, each group reading its active-run count every four
 * generations (for tools that cannot see kernels inside conditional graphs,
 * such as kernel profilers).  Results are identical. */
int adg_ctx_set_graphs(adg_ctx* ctx, int enable);

/* Launch geometry of adg_dock (no counterpart in the paper, whose kernels
 * have one fixed block shape per ligand).  The generation kernel runs one
 * individual per warp; per launch it chooses the warps per block and whether
 * the ligand's pair tables are copied into shared memory once per block or
 * read through L1, which sets how many warps stay resident per SM.
 *   ADG_GEO_HEURISTIC: one fixed rule (stage the ligand when it fits beside
 *     at least four warps, two blocks per SM), ligands grouped by atoms per
 *     lane (1..4, i.e. up to 32, 64, 96, 128 atoms).
 *   ADG_GEO_TUNED (default): the first time a shape bucket (atoms per lane,
 *     local-search kind, pair slots rounded up to 256, ligand bytes rounded
 *     up to 8 KiB) is met, the library times the geometries that keep the
 *     most warps resident -- ligand staged, and ligand read through L1 -- on
 *     a probe batch of that ligand's poses (each warp evaluating its pose
 *     eight times, as in a local search) and keeps the faster one for the
 *     life of the context.  A dock call then groups its ligands by the
 *     geometry they got; each group is one graph, the groups run on
 *     concurrent streams.
 * Docking results do not depend on the geometry (every warp does the same
 * arithmetic in either form). */
enum { ADG_GEO_HEURISTIC = 0, ADG_GEO_TUNED = 1 };
int adg_ctx_set_geometry(adg_ctx* ctx, int mode);

/* One entry of a context's tuning table. */
typedef struct {
    int32_t apl;             /* atoms per lane                            */
    int32_t ls_method;       /* ADG_LS_*                                  */
    int32_t nslots_max;      /* bucket bound: pair slots                  */
    int32_t bytes_max;       /* bucket bound: ligand blob bytes           */
    int32_t staged;          /* chosen: ligand copied to shared memory    */
    int32_t warps_per_block; /* chosen                                    */
    int32_t blocks_per_sm;   /* resident blocks of the generation kernel  */
    int32_t ncand;           /* candidates timed (0 or 1: none timed)     */
    float us_per_eval[2];    /* probe time per evaluation: staged, L1     */
} adg_tuned_shape;
/* Copy up to `cap` entries of the tuning table to out; *n = entries held. */
int adg_ctx_tuned(adg_ctx* ctx, adg_tuned_shape* out, int cap, int* n);

/* Triage network (no counterpart in the paper, which has no learned part).
 * A three-layer perceptron nin -> 256 -> 256 -> 1 with ReLU: BF16 weights,
 * FP32 accumulation on the tensor cores, FP32 master weights trained by
 * Adam (beta 0.9 / 0.999, eps 1e-8) on the mean squared error of the
 * normalised target.  It predicts a ligand's final best docking energy from
 * adg_ligand_descriptors and the early part of adg_dock_traced's trace.
 * Parameters are packed as W1 [256][nin], b1 [256], W2 [256][256], b2 [256],
 * w3 [256], b3 [1] (adg_mlp_nparams floats).  Inputs are normalised inside
 * the network: x_hat = (x - mu) / sigma; predictions are returned as
 * y * sigma_y + mu_y.  Device pointers, asynchronous on the context's stream
 * unless stated. */
#define ADG_MLP_HIDDEN 256
#define ADG_MLP_NIN_MAX 32
typedef struct adg_mlp adg_mlp;
/* Number of packed parameters for nin inputs (ADG_EINVAL outside 1..32). */
int adg_mlp_nparams(int nin);
/* He-uniform weights from `seed`, zero biases, mu = 0, sigma = 1.  Synchronous. */
int adg_mlp_create(adg_ctx* ctx, int nin, uint64_t seed, adg_mlp** out);
int adg_mlp_destroy(adg_mlp* mlp);
/* FP32 master parameters to / from host memory (synchronous); setting them
 * also clears the Adam state. */
int adg_mlp_get_params(adg_ctx* ctx, const adg_mlp* mlp, float* out);
int adg_mlp_set_params(adg_ctx* ctx, adg_mlp* mlp, const float* in);
/* Normalisation (host arrays of nin floats; every sigma > 0). */
int adg_mlp_set_norm(adg_mlp* mlp, const float* mu, const float* sigma, float mu_y, float sigma_y);
/* y[b] = prediction for x[b] (x: [B][nin], y: [B]). */
int adg_mlp_forward(adg_ctx* ctx, const adg_mlp* mlp, const float* x, int B, float* y);
/* Engine of adg_mlp_forward, adg_mlp_grad, adg_mlp_train_step and
 * adg_mlp_fit: ADG_MLP_TCGEN05 (default) -- persistent CTAs over 128-row
 * tiles, tcgen05.mma with FP32 accumulators in tensor memory (training: the
 * forward with dh2, dh1 = dh2 W2 with W2^T staged, and the weight gradients
 * with the batch as the K dimension); ADG_MLP_MMA_SYNC -- warp-level
 * m16n8k16 MMAs over 32-row tiles.  Same numerics (BF16 operands and stored
 * x_hat, h1, dh2, dh1; FP32 accumulation, h2 and biases); each engine's
 * training is bit-reproducible (every sum has a fixed order). */
enum { ADG_MLP_MMA_SYNC = 0, ADG_MLP_TCGEN05 = 1 };
int adg_mlp_set_engine(adg_mlp* mlp, int engine);
/* Synchronous: ADG_ETIMEOUT if a bounded wait of a tcgen05 kernel expired
 * since the last check (forward: the rows of the tiles concerned were written
 * as NaN; training: those tiles added nothing to the gradient), else ADG_OK. */
int adg_mlp_check(adg_ctx* ctx, adg_mlp* mlp);
/* Bound, in nanoseconds, of each wait of the tcgen05 kernels (forward and
 * training) on their tensor-core MMAs (default 1e9; 0 = test the barrier once
 * and give up if the MMAs are not done).  A wait that gives up sets the
 * status adg_mlp_check reports (forward: the rows of that tile become NaN;
 * training: the tile adds nothing); every kernel still waits for each MMA it
 * issued, under its own 1 s bound, before it frees its tensor memory, so the
 * context stays usable.  The paper has no counterpart: this
 * is the failure-detection path of the device waits, exposed so that it can
 * be exercised.  ns < 0: ADG_EINVAL. */
int adg_mlp_set_wait_ns(adg_mlp* mlp, long long ns);
/* Gradient of the batch loss (1/B) sum_b (y_b - (t_b - mu_y)/sigma_y)^2 with
 * respect to the packed parameters into grad [nparams], and the loss into
 * *loss (nullable); idx (nullable) selects rows of x and t.  No update. */
int adg_mlp_grad(adg_ctx* ctx, adg_mlp* mlp, const float* x, const float* t, const int* idx, int B, float* grad,
                 float* loss);
/* The same gradient followed by one Adam step with learning rate lr. */
int adg_mlp_train_step(adg_ctx* ctx, adg_mlp* mlp, const float* x, const float* t, const int* idx, int B, float lr,
                       float* loss);
/* `epochs` passes over n rows in minibatches of `batch`, rows shuffled each
 * epoch (seeded), one Adam step per minibatch.  epoch_loss: host [epochs]
 * (nullable), the mean loss seen during each epoch.  Synchronous. */
int adg_mlp_fit(adg_ctx* ctx, adg_mlp* mlp, const float* x, const float* t, int n, int batch, int epochs, float lr,
                uint64_t seed, float* epoch_loss);

/* Docking without allocation.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate memory -- a host application whose
 * own allocator owns all device memory and does not let libraries allocate
 * behind its back, or a latency-critical loop in which cudaMalloc/cudaFree
 * (which may synchronize the device) would stall other work.
 *
 * adg_dock_noalloc docks one ligand like adg_dock with nlig = 1 and no trace,
 * and allocates nothing: no cudaMalloc, no cudaFree, no host heap, no
 * allocating library call.  Its working memory is one device array of
 * ADG_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until
 * the process exits.  Limits: p->nrun <= ADG_NOALLOC_MAX_RUNS and
 * p->nrun * p->pop_size <= ADG_NOALLOC_MAX_INDIVIDUALS; larger requests return
 * ADG_ETOOBIG and touch nothing.
 *   rec, lig: built beforehand with adg_receptor_create / adg_ligand_create
 *   out:      host, caller-allocated [p->nrun], filled as by adg_dock
 *   stream:   cudaStream_t to run on (NULL: the legacy default stream)
 * The first call on a device looks up the array's device address there
 * (cudaGetSymbolAddress).  CUDA loads the code module holding the array
 * lazily, so the GPU reserves the array's memory at that lookup, not when the
 * library is loaded: make the first call on each device at set-up, before
 * the application's own allocator takes the device's memory, and before any
 * stream capture.  The call runs on rec's device and restores the caller's
 * current device before it returns.  Every call reuses the same array and
 * clears what must start at zero; calls whose GPU work overlaps (on
 * different streams or host threads) race on it and must be serialized by
 * the caller.  Returns when the results are in `out`. */
#define ADG_NOALLOC_SCRATCH_BYTES (4u << 20)
#define ADG_NOALLOC_MAX_RUNS 128
#define ADG_NOALLOC_MAX_INDIVIDUALS 16384
int adg_dock_noalloc(const adg_receptor* rec, const adg_ligand* lig, const adg_search_params* p, adg_result* out,
                     void* stream);

/* The schedule adg_ligand_create builds for a ligand, reported without a
 * device or a context: pair-loop steps (slots per lane; the kernel runs two
 * per step) and force-gather groups per lane, the empty slots, and the
 * shared-memory wavefronts one energy+gradient evaluation of the scoring
 * kernel spends in the pair loop (pair records, row and partner coordinates,
 * c_p stores, row-end force stores) and in the force gather (entries, c_p,
 * partner coordinates, the per-atom flush), modelled from the schedule: a
 * 16-byte access by a warp runs as four quarter-warp phases, each taking as
 * many wavefronts as the most distinct 16-byte words on one of its eight bank
 * groups; a 4-byte access takes as many as the most distinct words on one of
 * the 32 banks; lanes on the same word share it.  *_ideal: the same accesses
 * without bank conflicts.  Same validation and error codes as
 * adg_ligand_create; out: host, caller-allocated. */
typedef struct adg_schedule_stats {
    int32_t natoms, npairs;
    int32_t nsteps;       /* pair slots per lane */
    int32_t gsteps;       /* force-gather groups of four entries per lane */
    int32_t empty_slots;  /* 32 * nsteps - npairs, at least 1 */
    int32_t pair_wavefronts, pair_wavefronts_ideal;
    int32_t gather_wavefronts, gather_wavefronts_ideal;
} adg_schedule_stats;
int adg_ligand_schedule(const adg_forcefield* ff, const adg_ligand_desc* d, adg_schedule_stats* out);

/* Philox4x32-10 (Salmon et al., SC'11) on the device: out[4i..4i+3] =
 * Philox(counter ctr[4i..4i+3], key = (key & 0xffffffff, key >> 32)).
 * ctr and out: device, 4*n uint32, each 16-byte aligned (ADG_EINVAL otherwise). */
int adg_philox(adg_ctx* ctx, const uint32_t* ctr, int n, uint64_t key, uint32_t* out);

/* Measured throughput of the units that bound one scoring evaluation (the
 * roofline terms of the evaluation: FP32 flops, special-function results for
 * the pair terms' exp / rsqrt / reciprocal, and random gathers of the
 * L2-resident maps).  Each probe is one launch of 8 blocks of 256 threads
 * per SM, timed with CUDA events on the context's stream after one untimed
 * launch; about 20 ms of GPU time in all.  Allocates and frees an 8 MiB
 * device buffer.  out: host, caller-allocated.  Returns ADG_EINVAL on a null
 * argument, ADG_ECUDA (text in adg_ctx_last_error) on a CUDA failure. */
typedef struct adg_peaks {
    double fp32_tflops;        /* the larger of the two FMA probes; FMA = 2 flops */
    double fp32_scalar_tflops; /* 16 independent scalar FMA chains per thread */
    double fp32x2_tflops;      /* 8 independent two-wide FMA chains per thread */
    double mufu_gops;          /* ex2.approx results per second, 1e9 */
    double mufu_rsqrt_gops;    /* rsqrt.approx results per second, 1e9 */
    double l2_gather_gbs;      /* 16-byte random loads over gather_bytes, 1e9 bytes per second */
    int64_t gather_bytes;      /* size of the gathered buffer */
    int32_t sms;               /* multiprocessors */
    int32_t sm_clock_mhz;      /* maximum SM clock the device reports */
} adg_peaks;
int adg_probe_peaks(adg_ctx* ctx, adg_peaks* out);

#ifdef __cplusplus
}
#endif

#endif /* ADG_H */
