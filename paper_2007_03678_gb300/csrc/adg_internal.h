// adg_internal.h -- layouts shared by the host half (adg_api.cu) and the
// device half (adg_kernels.cu) of libadg.so.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <utility>
#include <vector>

#include "adg.h"

namespace adg {

constexpr int kMaxAtoms = ADG_MAX_ATOMS;
constexpr int kMaxTors = ADG_MAX_TORS;
constexpr int kGeneStride = 24;  // population rows are padded to 24 floats (>= 7 + 16)
constexpr int kMaxWarpsPerBlock = 12;

// Per-warp shared memory (floats): xyz[na + 1] (posed atoms, then a pad atom
// at the origin with zero charge), f[na + 1] (then a sink slot) and pm[na]
// (float4 each), the fragment transforms W[52] (float4, three rows per
// fragment), genes, cand and best [32 each], then c[nslots] (the pair scalars
// (dE/dr)/r).  na = 32 * atoms-per-lane.
__host__ __device__ inline size_t warp_smem_floats(int na, int nslots) { return (size_t)12 * na + 312 + nslots; }

// Launch geometry of one warp-per-individual kernel launch.  The block's
// dynamic shared memory holds a copy of its ligand's blob (lig_bytes) and
// then one region per warp.
struct Geo {
    int apl;           // atoms per lane (1, 2, 3, 4)
    int na;            // 32 * apl
    int nslots;        // largest pair-slot count of the launched ligands
    int wpb;           // warps per block
    size_t lig_bytes;  // largest ligand blob of the launch (0: read the ligand from global memory)
    size_t smem;       // dynamic shared memory per block (bytes)
};

// Ligand as the kernels read it: one POD blob in device memory.
// Atoms are kept in an internal depth-first order of the rigid-fragment tree
// (root fragment first, each fragment followed by its subtree), so the atoms
// moved by torsion k are the contiguous range [slo[k], shi[k]).  Torsions are
// indexed by their genotype index k (theta_k = genes[7 + k]); fragment f > 0
// hangs from fragment fpar[f] on torsion ftor[f], at depth flev[f].
struct LigandDev {
    int natoms, ntors, npairs, nsteps;   // nsteps: pair slots per lane (even)
    int gsteps;                          // force-gather groups per lane
    int nfrag, maxlev;                   // fragments (ntors + 1) and the deepest level
    // the blob: this header, then the pair and gather arrays at these byte offsets
    int blob_bytes, off_pk, off_gent;
    float cx, cy, cz;                    // reference centroid
    // scoring constants (from the force field)
    float e_cap, rmin2, ms_A, ms_B, ms_k, ms_lb, inv_2s2, inv_s2, k_out;
    float wq;                            // w_elec * Coulomb constant: cq = wq q_i q_j
    // Atom index: the atom at depth-first position a (fragment after
    // fragment, each followed by its subtree) has index (a % apl) * 32 + a / apl,
    // so lane l holds positions apl l .. apl l + apl - 1 at indices l, l + 32,
    // ...; the indices of positions >= natoms are unused.  Every per-atom array
    // here and in shared memory, and every atom in the pair and gather
    // programs, uses the index.
    int apl;                             // atoms per lane of this layout (1-4)
    int last_idx;                        // index of position natoms - 1
    float4 ref[kMaxAtoms];               // reference x, y, z and charge q
    int tf[kMaxAtoms];                   // map type | fragment << 8
    int old_of_new[kMaxAtoms];           // the caller's index of each atom
    int ta[kMaxTors], tb[kMaxTors];      // torsion k's bond atoms (a on the root side)
    int hi_idx[kMaxTors], lo_idx[kMaxTors];  // torsion k moves positions [lo, hi): indices of hi - 1 and lo - 1 (-1: lo = 0)
    float4 tpt[kMaxTors];                // reference position of atom a
    float4 tax[kMaxTors];                // reference unit axis a -> b
    int fpar[kMaxTors + 1], ftor[kMaxTors + 1], flev[kMaxTors + 1];
};

// Intramolecular pairs, lane-interleaved: slot (step, lane) = step * 32 + lane,
// 16 bytes per slot, (c12, cm, cd, ij as bits), stored for two-slot steps:
// slots a = 2t * 32 + lane and b = a + 32 hold pk[a] = (c12_a, c12_b, cm_a,
// cm_b) and pk[b] = (cd_a, cd_b, ij_a, ij_b), with
// ij = i | j << 16 | kPairOwned | kPairRowEnd | kPairRowStart | kPairHB |
// target << 24, i < 256.  Atom i is the same for a whole row, so a lane reads
// its coordinates only at the row's first slot.  An empty slot has zero
// coefficients and no row-end flag; its row atom is the pad atom na (read at
// the lane's first empty slot, kPairRowStart), whose zero charge makes cq
// vanish too, so an empty slot adds exactly 0 to the energy and has c_p = 0.
// With m = 10 for H-bond pairs (kPairHB) and 6 otherwise, and cq = wq q_i q_j
// from the charges the posed coordinates carry in .w:
// E_pair = min(c12 r^-12 - cm r^-m, e_cap) + cq / (eps(r) r) + cd exp(-r^2/(2 s^2)).
// Forces.  Most pairs are owned by atom i: the pairs a lane runs are grouped
// into rows, one row per owning atom, each row on one lane only, so the lane
// sums c_p (x_i - x_j) in registers and stores it to f[target] at the row's
// last slot (kPairRowEnd), target = i.  A pair no row could take runs as a
// row of its own (kPairOwned clear) whose target is 32 * atoms-per-lane: the
// sink slot f[na] past the atoms, never read, so the kernel sums every slot
// the same way.  Everything else -- the partner side of owned pairs, and
// both sides of the unowned pairs -- goes through the force
// gather: after the pair pass has stored c_p of every slot, lane l runs
// gsteps groups of four entries gent[(k * 32 + l) * 4 + q] (one 16-byte load) = partner |
// atom << 7 | slot << 14 (one atom per group; bit 31 on the last entry of
// the atom's last group; lists padded with entries on an empty slot, c_p = 0,
// whose partner is any posed atom, and all-zero groups at the end), sums c_p
// and c_p x_partner over the atom's entries and at its last group stores both
// sums (pm[atom], zero for atoms without entries); the force scan adds
// x_atom sum c_p - sum c_p x_partner to the atom's force.  Every ligand has
// at least one empty slot.
constexpr int kPairOwned = 1 << 15;
constexpr int kPairRowEnd = 1 << 14;
constexpr int kPairRowStart = 1 << 13;  // first slot of a row: (re)load atom i's coordinates
constexpr int kPairHB = 1 << 12;        // 12-10 H-bond pair (else 12-6)
struct PairsDev {
    const float4* pk;
    const uint32_t* gent;
};

struct LigandRef {
    const LigandDev* hdr;
    PairsDev pairs;
};

// Receptor maps, packed per ligand atom type t as one 32-byte record per node
// holding both x-corners of the cell edge that starts there:
// (M_t, M_elec, M_desolv, 0) at (x, y, z) and at (x + 1, y, z) (the last
// node of a row repeats itself), so a trilinear lookup is four 32-byte loads.
struct MapsDev {
    const float4* packed;  // [7][nz][ny][nx][2]
    int nx, ny, nz;
    float ox, oy, oz;      // origin
    float h, inv_h;
    float hx, hy, hz;      // upper corner of the box
};

struct SearchDev {
    int nrun, pop, nev, max_gen, ls_method, ls_max_iters, elitism;
    uint32_t thr_ls, thr_cross, thr_mut, thr_tour;  // probability thresholds floor(p * 2^24)
    float sw_rho0, sw_rho_min, sw_expand, sw_contract;
    int sw_succ, sw_fail;
    float sw_scale_t, sw_scale_rot, sw_scale_tors;
    float ad_rho, ad_eps;
    float mut_t, mut_rot, mut_tors;
    uint32_t key0, key1;
    int autostop;
    float stopstd;
};

struct DockDev {
    const LigandRef* ligs;     // [nlig]
    const uint32_t* lig_id;    // Philox counter word 0 per ligand
    int nlig;
    int run0;                  // run index of this launch's first run (its runs are run0 .. run0 + nrun - 1)
    float* pop_genes[2];       // [nlig*nrun][pop][kGeneStride], double-buffered by generation parity
    float* pop_e[2];           // [nlig*nrun][pop]
    unsigned long long* evals; // [nlig*nrun]
    int* gen_done;             // [nlig*nrun]
    float* best_hist;          // [nlig*nrun][10] best energy of the last 10 generations (ring)
    int* stopped;              // [nlig*nrun] autostop fired
    float* best_trace;         // optional [nlig*nrun][best_trace_len]: best energy after generations 1..len
    int best_trace_len;
    // optional trace (one ligand): decisions [nrun][ngen][pop][12], genes [nrun][ngen][pop][kGeneStride], e
    int trace_ngen;
    int* tr_dec;
    float* tr_genes;
    float* tr_e;
};

struct ResultDev {
    float best_energy;
    int generations;
    long long evals;
    float genes[kGeneStride];
    float xyz[3 * kMaxAtoms];
};

// Launchers (adg_kernels.cu).  All asynchronous on `st`; return cudaGetLastError().
cudaError_t launch_maps_build(cudaStream_t st, const adg_forcefield& ff, const adg_grid_desc& g, int nrec,
                              const float4* rec_xyzq, const int* rec_type, float* maps_out);
cudaError_t launch_pack_maps(cudaStream_t st, const float* maps, const adg_grid_desc& g, float4* packed);
Geo make_geo(int apl, int nslots, size_t lig_bytes);
// The same shape with the ligand staged in shared memory or not and `wpb`
// warps per block (no fitting rule applied; smem may exceed what a block can have).
Geo make_geo_explicit(int apl, int nslots, size_t lig_bytes, bool staged, int wpb);
// Resident blocks per SM of the generation kernel for local search `ls` at
// geometry g (0: the geometry cannot launch).
int geo_blocks_per_sm(const Geo& g, int ls);
// The warps per block that keep the most warps of the generation kernel
// resident for a shape, staged or not; returns that warp count (0: none launches).
int geo_best(int apl, int nslots, size_t lig_bytes, bool staged, int ls, Geo* out);
// Launch geometries worth timing for a shape: for the ligand staged in shared
// memory and for it read through L1, the warps-per-block counts that keep the
// most warps resident.  Writes up to `cap` entries, returns how many.
int geo_candidates(int apl, int nslots, size_t lig_bytes, int ls, Geo* out, int cap);
// Autotuning probe: npose random poses of a ligand with T torsions about the
// box centre (translation within +-spread), written as [npose][7+T].
cudaError_t launch_probe_genes(cudaStream_t st, const MapsDev& m, int T, int npose, float spread, uint32_t seed,
                               float* genes);
// Autotuning workload: every warp evaluates its pose `reps` times (with a
// small torsion change between evaluations), as a local search does, with
// (grad != 0) or without the gradient; energy[pose] receives the last value.
cudaError_t launch_tune(cudaStream_t st, const MapsDev& m, const LigandRef& l, const Geo& g, const float* genes,
                        int npose, int reps, int grad, float* energy);
// Several ligands' poses in one launch (adg_score_multi): device arrays
// over the launch's ligands and blocks; rows of genes / energy / grad are
// `stride` floats apart.
struct ScoreMultiDev {
    const LigandRef* ligs;  // [nlig]
    const int* blk_lig;     // [nblocks] ligand of each block
    const int* lig_blk0;    // [nlig] first block of each ligand
    const int* lig_row0;    // [nlig] first row of each ligand
    const int* lig_npose;   // [nlig]
    const int* lig_nblk;    // [nlig] blocks of each ligand
    int stride;
};
cudaError_t launch_score_multi(cudaStream_t st, const MapsDev& m, const ScoreMultiDev& j, int nblocks, const Geo& g,
                               const float* genes, float* energy, float* grad, int grad_kind);
cudaError_t launch_score(cudaStream_t st, const MapsDev& m, const LigandRef& l, const Geo& g, const float* genes,
                         int npose, float* energy, float* grad, int grad_kind);
cudaError_t launch_pose(cudaStream_t st, const LigandRef& l, const Geo& g, const float* genes, int npose, float* xyz);
cudaError_t launch_philox(cudaStream_t st, const uint32_t* ctr, int n, uint32_t k0, uint32_t k1, uint32_t* out);
cudaError_t launch_dock_init(cudaStream_t st, const MapsDev& m, const SearchDev& s, const DockDev& d, const Geo& g);
// gen_dev: NULL, or a device int holding the number of generations completed
// (the kernels then run generation *gen_dev + 1 in place of `gen`; used by
// generation loops that run inside a CUDA graph).
cudaError_t launch_dock_generation(cudaStream_t st, const MapsDev& m, const SearchDev& s, const DockDev& d,
                                   const Geo& g, int gen, const int* gen_dev = nullptr);
cudaError_t launch_dock_count_active(cudaStream_t st, const SearchDev& s, const DockDev& d, int gen, int* active,
                                     const int* gen_dev = nullptr);
cudaError_t launch_dock_loop_ctl(cudaStream_t st, cudaGraphConditionalHandle h, int* gen_dev, int* active);
cudaError_t launch_dock_finalize(cudaStream_t st, const MapsDev& m, const SearchDev& s, const DockDev& d,
                                 const Geo& g, ResultDev* out);
// Same, writing adg_result records (device memory) instead of ResultDev.
cudaError_t launch_dock_finalize_abi(cudaStream_t st, const MapsDev& m, const SearchDev& s, const DockDev& d,
                                     const Geo& g, adg_result* out);

}  // namespace adg

// Handles of the C ABI (opaque to callers).
struct adg_receptor {
    adg_ctx* ctx = nullptr;  // creator; not dereferenced by adg_receptor_destroy
    int device = 0;
    adg_grid_desc grid{};
    float4* packed = nullptr;
    adg::MapsDev maps{};
};

struct adg_ligand {
    adg_ctx* ctx = nullptr;  // creator; not dereferenced by adg_ligand_destroy
    int device = 0;
    void* blob = nullptr;  // LigandDev followed by the pair arrays
    adg::LigandRef ref{};
    int natoms = 0, ntors = 0, npairs = 0, apl = 1, sum_moving = 0, nslots = 0;
    size_t bytes = 0;
    float desc[ADG_NDESC] = {};  // adg_ligand_descriptors
    int64_t stream_id = -1;      // adg_ligand_set_stream_id
};

// The context: device, stream, reusable device memory and counters.
struct adg_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string last_error;
    void* arena = nullptr;
    size_t arena_bytes = 0;
    int* host_active = nullptr;  // pinned
    // measurement
    bool timing = false;
    adg_stats stats{};
    std::vector<cudaEvent_t> ev_free;                       // reusable events
    std::vector<cudaStream_t> class_streams;  // extra streams for concurrent ligand groups
    bool use_graphs = true;  // adg_ctx_set_graphs
    // launch geometry of adg_dock
    int geo_mode = ADG_GEO_TUNED;
    std::map<uint32_t, adg_tuned_shape> tuned;  // by shape bucket
    void* tune_buf = nullptr;                    // probe poses and energies
    size_t tune_bytes = 0;
    // adg_score_multi's block -> ligand tables: the last upload, kept while
    // the next call's tables are the same bytes
    std::vector<char> multi_host;
    void* multi_dev = nullptr;
    size_t multi_cap = 0;
};
