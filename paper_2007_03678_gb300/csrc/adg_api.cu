// adg_api.cu -- host half of libadg.so: the C ABI declared in include/adg.h.
//
// Holds the context (device, stream, a grow-only device arena reused across
// dock calls: the paper's context and memory reuse, Sec. 2.2.3), the
// resident receptor (maps uploaded once, Sec. 2.2.3), the ligand
// preprocessing (torsion tree, intramolecular pair list and its lane
// schedule) and the generation loop of adg_dock.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "adg_internal.h"

using namespace adg;

namespace adg {
void pair_coefs(const adg_forcefield& ff, int ti, int tj, float* c12, float* c6, float* c10);
}


namespace {

int cuda_fail(adg_ctx* ctx, cudaError_t e, const char* what)
{
    if (ctx) ctx->last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return ADG_ECUDA;
}

#define CK(ctx, call)                                        \
    do {                                                     \
        cudaError_t _e = (call);                             \
        if (_e != cudaSuccess) return cuda_fail(ctx, _e, #call); \
    } while (0)

int apl_for(int natoms) { return (natoms + 31) / 32; }  // atoms per lane, 1..4

uint32_t prob_threshold(float p)
{
    if (p <= 0.f) return 0u;
    if (p >= 1.f) return 16777216u;
    return (uint32_t)floor((double)p * 16777216.0);
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int check_grid(const adg_grid_desc* g)
{
    if (!g) return ADG_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (g->n[a] < 2) return ADG_EGRID;
    if (!(g->spacing > 0.f)) return ADG_EGRID;
    return ADG_OK;
}

cudaError_t take_event(adg_ctx* ctx, cudaEvent_t* ev)
{
    if (!ctx->ev_free.empty()) {
        *ev = ctx->ev_free.back();
        ctx->ev_free.pop_back();
        return cudaSuccess;
    }
    return cudaEventCreate(ev);
}

}  // namespace

extern "C" {

const char* adg_strerror(int code)
{
    switch (code) {
    case ADG_OK: return "ok";
    case ADG_EINVAL: return "invalid argument (null pointer or bad size)";
    case ADG_ETYPE: return "atom type outside 0..6";
    case ADG_ETOOBIG: return "ligand exceeds ADG_MAX_ATOMS atoms or ADG_MAX_TORS torsions";
    case ADG_EGRID: return "grid needs at least 2 points per axis and a positive spacing";
    case ADG_ECUDA: return "CUDA runtime error";
    case ADG_ETIMEOUT: return "bounded device wait expired";
    case ADG_ENOMEM: return "out of memory";
    case ADG_ETOPO: return "bonds are not one tree or a torsion is not a bond";
    default: return "unknown error";
    }
}

void adg_search_params_default(adg_search_params* p)
{
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->nrun = 10;
    p->pop_size = 150;
    p->nev = 2500000;
    p->max_gen = 27000;
    p->ls_method = ADG_LS_SOLIS_WETS;
    p->ls_max_iters = 300;
    p->elitism = 1;
    p->ls_rate = 1.f;
    p->crossover_rate = 0.8f;
    p->mutation_rate = 0.02f;
    p->tournament_rate = 0.6f;
    p->sw_rho0 = 1.f;
    p->sw_rho_min = 0.01f;
    p->sw_expand = 2.f;
    p->sw_contract = 0.5f;
    p->sw_succ = 4;
    p->sw_fail = 4;
    p->sw_scale_t = 1.f;
    p->sw_scale_rot = 0.5f;
    p->sw_scale_tors = 0.5f;
    p->ad_rho = 0.8f;
    p->ad_eps = 0.01f;
    p->mut_t = 2.f;
    p->mut_rot = 1.57079632679490f;
    p->mut_tors = 1.57079632679490f;
    p->seed = 42;
    p->lig_id = 0;
    p->autostop = 0;
    p->stopstd = 0.15f;
}

int adg_ctx_create(adg_ctx** out, int device, void* stream)
{
    if (!out) return ADG_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return ADG_EINVAL;
    adg_ctx* c = new (std::nothrow) adg_ctx();
    if (!c) return ADG_ENOMEM;
    c->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) {
        if (stream) {
            c->stream = (cudaStream_t)stream;
        } else {
            e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
            c->own_stream = true;
        }
    }
    if (e == cudaSuccess) e = cudaMallocHost(&c->host_active, sizeof(int) * 4);
    if (e != cudaSuccess) {
        if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
        delete c;
        return ADG_ECUDA;
    }
    *out = c;
    return ADG_OK;
}

int adg_ctx_destroy(adg_ctx* ctx)
{
    if (!ctx) return ADG_EINVAL;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (auto ev : ctx->ev_free) cudaEventDestroy(ev);
    for (auto s2 : ctx->class_streams) {
        cudaStreamSynchronize(s2);
        cudaStreamDestroy(s2);
    }
    if (ctx->arena) cudaFree(ctx->arena);
    if (ctx->tune_buf) cudaFree(ctx->tune_buf);
    if (ctx->multi_dev) cudaFree(ctx->multi_dev);
    if (ctx->host_active) cudaFreeHost(ctx->host_active);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return ADG_OK;
}

int adg_sync(adg_ctx* ctx)
{
    if (!ctx) return ADG_EINVAL;
    CK(ctx, cudaSetDevice(ctx->device));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return ADG_OK;
}

const char* adg_ctx_last_error(const adg_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

int adg_ctx_set_timing(adg_ctx* ctx, int enable)
{
    if (!ctx) return ADG_EINVAL;
    ctx->timing = enable != 0;
    return ADG_OK;
}

int adg_ctx_set_graphs(adg_ctx* ctx, int enable)
{
    if (!ctx) return ADG_EINVAL;
    ctx->use_graphs = enable != 0;
    return ADG_OK;
}

int adg_ctx_set_geometry(adg_ctx* ctx, int mode)
{
    if (!ctx || (mode != ADG_GEO_HEURISTIC && mode != ADG_GEO_TUNED)) return ADG_EINVAL;
    ctx->geo_mode = mode;
    return ADG_OK;
}

int adg_ctx_tuned(adg_ctx* ctx, adg_tuned_shape* out, int cap, int* n)
{
    if (!ctx || !n || cap < 0 || (cap > 0 && !out)) return ADG_EINVAL;
    *n = (int)ctx->tuned.size();
    int k = 0;
    for (const auto& kv : ctx->tuned) {
        if (k >= cap) break;
        out[k++] = kv.second;
    }
    return ADG_OK;
}

int adg_ctx_stats(adg_ctx* ctx, adg_stats* out, int reset)
{
    if (!ctx || !out) return ADG_EINVAL;
    *out = ctx->stats;
    if (reset) ctx->stats = adg_stats{};
    return ADG_OK;
}

int adg_maps_build(adg_ctx* ctx, const adg_forcefield* ff, const adg_grid_desc* grid, int nrec, const float* rec_xyz,
                   const int32_t* rec_type, const float* rec_q, float* maps_out)
{
    if (!ctx || !ff || !rec_xyz || !rec_type || !rec_q || !maps_out || nrec <= 0) return ADG_EINVAL;
    int rc = check_grid(grid);
    if (rc) return rc;
    std::vector<float4> xq(nrec);
    for (int i = 0; i < nrec; ++i) {
        if (rec_type[i] < 0 || rec_type[i] >= ADG_NTYPES) return ADG_ETYPE;
        xq[i] = make_float4(rec_xyz[3 * i], rec_xyz[3 * i + 1], rec_xyz[3 * i + 2], rec_q[i]);
    }
    CK(ctx, cudaSetDevice(ctx->device));
    float4* d_xq = nullptr;
    int* d_t = nullptr;
    CK(ctx, cudaMallocAsync(&d_xq, sizeof(float4) * nrec, ctx->stream));
    CK(ctx, cudaMallocAsync(&d_t, sizeof(int) * nrec, ctx->stream));
    CK(ctx, cudaMemcpyAsync(d_xq, xq.data(), sizeof(float4) * nrec, cudaMemcpyHostToDevice, ctx->stream));
    CK(ctx, cudaMemcpyAsync(d_t, rec_type, sizeof(int) * nrec, cudaMemcpyHostToDevice, ctx->stream));
    CK(ctx, launch_maps_build(ctx->stream, *ff, *grid, nrec, d_xq, d_t, maps_out));
    ctx->stats.kernel_launches += 1;
    CK(ctx, cudaFreeAsync(d_xq, ctx->stream));
    CK(ctx, cudaFreeAsync(d_t, ctx->stream));
    // the host vectors are read by the copies above: wait before they go out of scope
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return ADG_OK;
}

int adg_receptor_create(adg_ctx* ctx, const adg_grid_desc* grid, const float* maps, int maps_on_device,
                        adg_receptor** out)
{
    if (!ctx || !maps || !out) return ADG_EINVAL;
    *out = nullptr;
    int rc = check_grid(grid);
    if (rc) return rc;
    CK(ctx, cudaSetDevice(ctx->device));
    const long npt = (long)grid->n[0] * grid->n[1] * grid->n[2];
    adg_receptor* r = new (std::nothrow) adg_receptor();
    if (!r) return ADG_ENOMEM;
    r->ctx = ctx;
    r->device = ctx->device;
    r->grid = *grid;
    cudaError_t e = cudaMalloc(&r->packed, 2 * sizeof(float4) * ADG_NTYPES * npt);
    if (e != cudaSuccess) {
        delete r;
        return cuda_fail(ctx, e, "cudaMalloc(packed maps)");
    }
    const float* src = maps;
    float* tmp = nullptr;
    if (!maps_on_device) {
        e = cudaMallocAsync(&tmp, sizeof(float) * ADG_NMAPS * npt, ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(tmp, maps, sizeof(float) * ADG_NMAPS * npt, cudaMemcpyHostToDevice, ctx->stream);
        src = tmp;
    }
    if (e == cudaSuccess) e = launch_pack_maps(ctx->stream, src, *grid, r->packed);
    ctx->stats.kernel_launches += 1;
    if (tmp) cudaFreeAsync(tmp, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        cudaFree(r->packed);
        delete r;
        return cuda_fail(ctx, e, "receptor upload");
    }
    MapsDev& m = r->maps;
    m.packed = r->packed;
    m.nx = grid->n[0];
    m.ny = grid->n[1];
    m.nz = grid->n[2];
    m.ox = grid->origin[0];
    m.oy = grid->origin[1];
    m.oz = grid->origin[2];
    m.h = grid->spacing;
    m.inv_h = 1.f / grid->spacing;
    m.hx = grid->origin[0] + (grid->n[0] - 1) * grid->spacing;
    m.hy = grid->origin[1] + (grid->n[1] - 1) * grid->spacing;
    m.hz = grid->origin[2] + (grid->n[2] - 1) * grid->spacing;
    *out = r;
    return ADG_OK;
}

int adg_receptor_destroy(adg_receptor* rec)
{
    if (!rec) return ADG_EINVAL;
    // independent of the context, which may already be gone; cudaFree waits
    // for work that still uses the memory
    cudaSetDevice(rec->device);
    cudaFree(rec->packed);
    delete rec;
    return ADG_OK;
}

}  // extern "C"

namespace {

// The distinct words one shared-memory access reads, by bank: a 16-byte
// access by a quarter-warp (8 groups of four banks) or a 4-byte access by a
// warp (32 banks).  cost(w) = the wavefronts reading w as well would add.
template <int BANKS>
struct WordSet {
    int words[32];
    int n = 0, mx = 0;
    int cnt[BANKS] = {};
    bool has(int w) const
    {
        for (int k = 0; k < n; ++k)
            if (words[k] == w) return true;
        return false;
    }
    int cost(int w) const { return has(w) ? 0 : std::max(0, cnt[w % BANKS] + 1 - mx); }
    // ranks a choice: added wavefronts first, then a word already read (shared
    // for free) over a new one, then the fuller its bank would get
    int rank(int w) const { return has(w) ? 0 : 64 * cost(w) + 1 + cnt[w % BANKS]; }
    void add(int w)
    {
        if (has(w)) return;
        words[n++] = w;
        mx = std::max(mx, ++cnt[w % BANKS]);
    }
};

// Host-side plan of a ligand: the device header, the pair records and the
// force-gather program the scoring kernel runs, built without touching a
// device (adg_ligand_create uploads it; adg_ligand_schedule reports on it).
struct LigandPlan {
    LigandDev h;
    std::vector<uint4> pk;
    std::vector<uint32_t> gent;
    int nf = 0, sum_moving = 0;
};

// Local search on the force-gather program.  An atom's entries may sit at any
// position of the atom's groups (the sums do not depend on where), so two
// entries of one atom are swapped unless that raises the modelled wavefronts
// of the two positions' loads: the c_p words (one 4-byte load by the warp)
// and the partner coordinates (16-byte loads, quarter-warps).
// Padding entries (c_p = 0) may read any empty slot and any partner, and the
// entries of a lane past its atoms (never stored) any slot and any partner:
// each takes a word its load already reads where it can.  Deterministic (a
// fixed xorshift stream), `budget` proposed swaps.
constexpr long kGatherRefinePerEntry = 4;  // proposed swaps per gather entry

struct GatherRefine {
    std::vector<uint32_t>& gent;
    const int ngroups;
    const std::vector<char>& used;      // used[atom index]: a posed atom lives there
    const std::vector<int>& blk;        // [k * 32 + l]: the atom block of lane l's group k, -1 past its atoms
    const std::vector<char>& empty;     // empty[slot]: c_p of the slot is exactly 0
    int empty_of_bank[32];              // the lowest empty slot in each bank, -1 if none
    enum { REAL = 0, PAD = 1, FREE = 2 };
    std::vector<int> kind, cw, xw;      // per entry (k * 32 + l) * 4 + q

    GatherRefine(std::vector<uint32_t>& g, int ng, const std::vector<char>& u, const std::vector<int>& b,
                 const std::vector<char>& em)
        : gent(g), ngroups(ng), used(u), blk(b), empty(em)
    {
        for (int b = 0; b < 32; ++b) empty_of_bank[b] = -1;
        for (int s = 0; s < (int)em.size(); ++s)
            if (em[s] && empty_of_bank[s % 32] < 0) empty_of_bank[s % 32] = s;
        const size_t n = gent.size();
        kind.assign(n, REAL);
        cw.assign(n, 0);
        xw.assign(n, 0);
        for (size_t i = 0; i < n; ++i) {
            const uint32_t e = gent[i];
            cw[i] = (int)((e >> 14) & 0xffff);
            xw[i] = (int)(e & 127);
            if (blk[i / 4] < 0) kind[i] = FREE;
            else if (empty[cw[i]]) kind[i] = PAD;
        }
    }
    // modelled wavefronts of position q of group k; with `commit` the
    // flexible entries keep the words chosen for them.  Words are kept per
    // bank, so a membership test scans one bank; a flexible entry takes the
    // first word added (padding: the first empty slot added).
    int cost(int k, int q, bool commit)
    {
        int bw[32][32], cnt[32], mx = 0, tot = 0, first = -1, first_empty = -1;
        auto add = [&](int w, int banks, bool slot) {
            const int b = w % banks;
            for (int t = 0; t < cnt[b]; ++t)
                if (bw[b][t] == w) return;
            bw[b][cnt[b]++] = w;
            mx = std::max(mx, cnt[b]);
            if (first < 0) first = w;
            if (slot && first_empty < 0 && empty[w]) first_empty = w;
        };
        const size_t base = (size_t)k * 128 + q;
        for (int b = 0; b < 32; ++b) cnt[b] = 0;
        for (int l = 0; l < 32; ++l)
            if (kind[base + 4 * l] == REAL) add(cw[base + 4 * l], 32, true);
        for (int l = 0; l < 32; ++l) {
            const size_t i = base + 4 * l;
            if (kind[i] == REAL) continue;
            int w = kind[i] == FREE ? first : first_empty;
            if (w < 0) {
                if (kind[i] == FREE) w = 0;
                else {  // the lowest empty slot among the least filled banks that hold one
                    int best = 1 << 30;
                    for (int b = 0; b < 32; ++b) {
                        const int e = empty_of_bank[b];
                        if (e >= 0 && (cnt[b] < best || (cnt[b] == best && e < w))) {
                            best = cnt[b];
                            w = e;
                        }
                    }
                }
            }
            add(w, 32, true);
            if (commit) cw[i] = w;
        }
        tot += mx;
        for (int qd = 0; qd < 4; ++qd) {
            mx = 0;
            first = -1;
            for (int b = 0; b < 8; ++b) cnt[b] = 0;
            for (int l = qd * 8; l < qd * 8 + 8; ++l)
                if (kind[base + 4 * l] == REAL) add(xw[base + 4 * l], 8, false);
            for (int l = qd * 8; l < qd * 8 + 8; ++l) {
                const size_t i = base + 4 * l;
                if (kind[i] == REAL) continue;
                int w = first >= 0 ? first : 0;
                if (first < 0 && kind[i] == PAD) w = used[xw[i]] ? xw[i] : 0;
                add(w, 8, false);
                if (commit) xw[i] = w;
            }
            tot += mx;
        }
        return tot;
    }
    void run(long budget)
    {
        // each lane's blocks: first group and group count
        std::vector<std::vector<std::pair<int, int>>> blocks(32);
        for (int l = 0; l < 32; ++l)
            for (int k = 0; k < ngroups; ++k) {
                const int b = blk[(size_t)k * 32 + l];
                if (b < 0) continue;
                if (blocks[l].empty() || blocks[l].back().first + blocks[l].back().second != k ||
                    blk[(size_t)(k - 1) * 32 + l] != b)
                    blocks[l].push_back({k, 1});
                else
                    ++blocks[l].back().second;
            }
        uint32_t st = 0x9e3779b9u;
        auto rnd = [&](uint32_t n) {
            st ^= st << 13;
            st ^= st >> 17;
            st ^= st << 5;
            return (uint32_t)(((uint64_t)st * n) >> 32);
        };
        std::vector<int> cc((size_t)ngroups * 4);  // each position's current cost
        for (int k = 0; k < ngroups; ++k)
            for (int q = 0; q < 4; ++q) cc[(size_t)k * 4 + q] = cost(k, q, false);
        for (long it = 0; it < budget; ++it) {
            const int l = (int)rnd(32);
            if (blocks[l].empty()) continue;
            const auto& bk = blocks[l][rnd((uint32_t)blocks[l].size())];
            const int npos = 4 * bk.second;
            if (npos < 2) continue;
            const int p1 = (int)rnd(npos), p2 = (int)rnd(npos);
            const int k1 = bk.first + p1 / 4, q1 = p1 % 4, k2 = bk.first + p2 / 4, q2 = p2 % 4;
            if (k1 == k2 && q1 == q2) continue;  // the same position: nothing to swap
            const size_t i1 = ((size_t)k1 * 32 + l) * 4 + q1, i2 = ((size_t)k2 * 32 + l) * 4 + q2;
            const int before = cc[(size_t)k1 * 4 + q1] + cc[(size_t)k2 * 4 + q2];
            std::swap(kind[i1], kind[i2]);
            std::swap(cw[i1], cw[i2]);
            std::swap(xw[i1], xw[i2]);
            const int c1 = cost(k1, q1, false), c2 = cost(k2, q2, false);
            if (c1 + c2 > before) {
                std::swap(kind[i1], kind[i2]);
                std::swap(cw[i1], cw[i2]);
                std::swap(xw[i1], xw[i2]);
            } else {
                cc[(size_t)k1 * 4 + q1] = c1;
                cc[(size_t)k2 * 4 + q2] = c2;
            }
        }
    }
    void store()
    {
        for (int k = 0; k < ngroups; ++k)
            for (int q = 0; q < 4; ++q) cost(k, q, true);
        for (size_t i = 0; i < gent.size(); ++i) {
            const uint32_t keep = gent[i] & (0x7fu << 7 | 0x80000000u);  // atom and last-group bit stay with the position
            gent[i] = (kind[i] == FREE ? 0u : keep) | (uint32_t)xw[i] | ((uint32_t)cw[i] << 14);
        }
    }
};

int plan_ligand(const adg_forcefield* ff, const adg_ligand_desc* d, LigandPlan& pl)
{
    if (!ff || !d || !d->xyz || !d->type || !d->charge) return ADG_EINVAL;
    const int N = d->natoms, T = d->ntors;
    if (N < 1 || T < 0 || d->nbonds < 0) return ADG_EINVAL;
    if (N > ADG_MAX_ATOMS || T > ADG_MAX_TORS) return ADG_ETOOBIG;
    if ((d->nbonds > 0 && !d->bonds) || (T > 0 && !d->tors)) return ADG_EINVAL;
    if (d->root < 0 || d->root >= N) return ADG_EINVAL;
    for (int i = 0; i < N; ++i)
        if (d->type[i] < 0 || d->type[i] >= ADG_NTYPES) return ADG_ETYPE;
    for (int i = 0; i < 3 * N; ++i)
        if (!isfinite(d->xyz[i])) return ADG_EINVAL;
    // --- tree: adjacency, BFS from the root (parent, depth)
    if (d->nbonds != N - 1) return ADG_ETOPO;
    std::vector<std::vector<int>> adj(N);
    for (int b = 0; b < d->nbonds; ++b) {
        const int i = d->bonds[2 * b], j = d->bonds[2 * b + 1];
        if (i < 0 || j < 0 || i >= N || j >= N || i == j) return ADG_ETOPO;
        adj[i].push_back(j);
        adj[j].push_back(i);
    }
    std::vector<int> parent(N, -2), depth(N, 0), bfs;
    bfs.reserve(N);
    parent[d->root] = -1;
    bfs.push_back(d->root);
    for (size_t h = 0; h < bfs.size(); ++h)
        for (int v : adj[bfs[h]])
            if (parent[v] == -2) {
                parent[v] = bfs[h];
                depth[v] = depth[bfs[h]] + 1;
                bfs.push_back(v);
            }
    if ((int)bfs.size() != N) return ADG_ETOPO;
    // --- torsions: orient a -> b away from the root; moving set = subtree of b
    std::vector<int> ta(T), tb(T);
    std::vector<std::vector<char>> moving(T, std::vector<char>(N, 0));
    for (int k = 0; k < T; ++k) {
        int a = d->tors[2 * k], b = d->tors[2 * k + 1];
        if (a < 0 || b < 0 || a >= N || b >= N) return ADG_ETOPO;
        if (parent[b] == a) {
        } else if (parent[a] == b) {
            std::swap(a, b);
        } else {
            return ADG_ETOPO;
        }
        ta[k] = a;
        tb[k] = b;
        // atoms whose root path passes through b: walk up from each atom
        for (int i = 0; i < N; ++i) {
            for (int u = i; u >= 0; u = parent[u])
                if (u == b) {
                    moving[k][i] = 1;
                    break;
                }
        }
    }
    // --- rigid fragments (bonds that are not rotatable) and graph distances <= 3
    std::vector<int> frag(N, -1);
    auto is_rot = [&](int u, int v) {
        for (int k = 0; k < T; ++k)
            if ((ta[k] == u && tb[k] == v) || (ta[k] == v && tb[k] == u)) return true;
        return false;
    };
    int nf = 0;
    for (int s = 0; s < N; ++s) {
        if (frag[s] >= 0) continue;
        std::vector<int> st{s};
        frag[s] = nf;
        while (!st.empty()) {
            const int u = st.back();
            st.pop_back();
            for (int v : adj[u])
                if (frag[v] < 0 && !is_rot(u, v)) {
                    frag[v] = nf;
                    st.push_back(v);
                }
        }
        ++nf;
    }
    // --- fragment tree and the internal depth-first atom order: each fragment
    // is followed by its subtree, so the atoms a torsion moves are contiguous
    if (nf != T + 1) return ADG_ETOPO;
    std::vector<int> fpar(nf, -1), ftor(nf, -1);
    std::vector<std::vector<int>> fchild(nf);
    for (int k = 0; k < T; ++k) {
        const int cf = frag[tb[k]], pf = frag[ta[k]];
        if (cf == pf || ftor[cf] >= 0) return ADG_ETOPO;
        fpar[cf] = pf;
        ftor[cf] = k;
        fchild[pf].push_back(cf);
    }
    std::vector<int> fnew(nf, -1), forder, flev(nf, 0);
    {
        std::vector<int> st{frag[d->root]};
        while (!st.empty()) {
            const int f = st.back();
            st.pop_back();
            fnew[f] = (int)forder.size();
            forder.push_back(f);
            for (auto it = fchild[f].rbegin(); it != fchild[f].rend(); ++it) {
                flev[*it] = flev[f] + 1;
                st.push_back(*it);
            }
        }
    }
    if ((int)forder.size() != nf) return ADG_ETOPO;
    std::vector<int> nw(N, -1), old_of;  // caller index -> internal, internal -> caller
    std::vector<int> flo(nf), fhi(nf);   // atom range of each fragment (internal fragment index)
    for (int fi = 0; fi < nf; ++fi) {
        flo[fi] = (int)old_of.size();
        for (int i = 0; i < N; ++i)
            if (frag[i] == forder[fi]) {
                nw[i] = (int)old_of.size();
                old_of.push_back(i);
            }
        fhi[fi] = (int)old_of.size();
    }
    std::vector<int> send(nf);  // end of each fragment's subtree (atoms)
    for (int fi = nf - 1; fi >= 0; --fi) {
        send[fi] = fhi[fi];
        for (int c : fchild[forder[fi]]) send[fi] = std::max(send[fi], send[fnew[c]]);
    }
    std::vector<int> slo(T), shi(T);
    int maxlev = 0;
    for (int k = 0; k < T; ++k) {
        const int c = fnew[frag[tb[k]]];
        slo[k] = flo[c];
        shi[k] = send[c];
        for (int i = 0; i < N; ++i)
            if ((moving[k][i] != 0) != (nw[i] >= slo[k] && nw[i] < shi[k])) return ADG_ETOPO;
    }
    for (int f = 0; f < nf; ++f) maxlev = std::max(maxlev, flev[f]);
    std::vector<std::vector<char>> near(N, std::vector<char>(N, 0));
    for (int s = 0; s < N; ++s) {
        std::vector<int> dist(N, -1), q{s};
        dist[s] = 0;
        for (size_t h = 0; h < q.size(); ++h) {
            const int u = q[h];
            if (dist[u] == 3) continue;
            for (int v : adj[u])
                if (dist[v] < 0) {
                    dist[v] = dist[u] + 1;
                    q.push_back(v);
                }
        }
        for (int v : q) near[s][v] = 1;
    }
    // --- atom indices: position a of the depth-first order gets index
    // (a % apl) * 32 + a / apl, so each lane's atoms are consecutive positions
    // (the force scan then needs one warp scan per evaluation, not apl); the
    // pair and gather programs below work on indices
    const int apl = apl_for(N), na = 32 * apl;
    auto idx_of = [&](int a) { return (a % apl) * 32 + a / apl; };
    std::vector<int> src_of(na, -1);  // the caller's index of the atom at each index, -1 if unused
    for (int a = 0; a < N; ++a) src_of[idx_of(a)] = old_of[a];
    std::vector<std::pair<int, int>> pairs;  // atom indices
    for (int i = 0; i < N; ++i)
        for (int j = i + 1; j < N; ++j)
            if (frag[i] != frag[j] && !near[i][j]) {
                const int x = idx_of(nw[i]), y = idx_of(nw[j]);
                pairs.emplace_back(std::min(x, y), std::max(x, y));
            }
    const int P = (int)pairs.size();
    // --- lane schedule.  Rows: the not yet owned atom with the most
    // unscheduled pairs takes (up to a lane's share of) those pairs as its row,
    // first the pairs whose partner already owns a row (no row could take them
    // later).  A row runs on one lane, which keeps the owner's coordinates and
    // force in registers.  Pairs no row takes run as one-pair rows, unowned.
    std::vector<std::vector<int>> inc_p(na);  // pairs by atom
    for (int p = 0; p < P; ++p) {
        inc_p[pairs[p].first].push_back(p);
        inc_p[pairs[p].second].push_back(p);
    }
    struct Row {
        int owner;               // -1: one unowned pair
        std::vector<int> ps;     // pair ids
    };
    std::vector<Row> rows;
    std::vector<int> owner(P, -1);
    {
        std::vector<char> sched(P, 0), done(na, 0);
        std::vector<int> load(32, 0);
        const int share = (P + 31) / 32;
        for (;;) {
            const int lane = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            const int room = share - load[lane];
            if (room <= 0) break;
            int best = -1, best_n = 0;
            for (int pos = 0; pos < N; ++pos) {
                const int a2 = idx_of(pos);
                if (done[a2]) continue;
                int n2 = 0;
                for (int p : inc_p[a2]) n2 += !sched[p];
                if (n2 > best_n) { best = a2; best_n = n2; }
            }
            if (best < 0) break;
            Row r{best, {}};
            for (int p : inc_p[best])
                if (!sched[p] && done[pairs[p].first + pairs[p].second - best]) r.ps.push_back(p);
            for (int p : inc_p[best])
                if (!sched[p] && !done[pairs[p].first + pairs[p].second - best]) r.ps.push_back(p);
            r.ps.resize(std::min((int)r.ps.size(), room));
            for (int p : r.ps) {
                owner[p] = best;
                sched[p] = 1;
            }
            load[lane] += (int)r.ps.size();
            done[best] = 1;
            rows.push_back(r);
        }
        for (int p = 0; p < P; ++p)
            if (!sched[p]) rows.push_back(Row{-1, {p}});
    }
    // Rows to lanes, longest first to the least loaded lane; among those,
    // one whose quarter-warp holds no owner with the same atom index mod 8
    // (a 16-byte shared-memory load by eight lanes is conflict-free when their
    // atoms differ mod 8).
    std::vector<std::vector<int>> lane_rows(32);
    {
        std::vector<int> order(rows.size());
        for (size_t r = 0; r < rows.size(); ++r) order[r] = (int)r;
        std::stable_sort(order.begin(), order.end(),
                         [&](int x, int y) { return rows[x].ps.size() > rows[y].ps.size(); });
        std::vector<int> load(32, 0);
        std::vector<int> qres(4, 0);  // residues held per quarter (bit mask)
        for (int r : order) {
            const int m = *std::min_element(load.begin(), load.end());
            const int res = rows[r].owner >= 0 ? rows[r].owner % 8 : -1;
            int lane = -1;
            for (int l = 0; l < 32 && lane < 0; ++l)
                if (load[l] == m && (res < 0 || !(qres[l / 8] >> res & 1))) lane = l;
            if (lane < 0)
                for (int l = 0; l < 32 && lane < 0; ++l)
                    if (load[l] == m) lane = l;
            lane_rows[lane].push_back(r);
            load[lane] += (int)rows[r].ps.size();
            if (res >= 0) qres[lane / 8] |= 1 << res;
        }
    }
    int nsteps = 0;
    for (int l = 0; l < 32; ++l) {
        int n2 = 0;
        for (int r : lane_rows[l]) n2 += (int)rows[r].ps.size();
        nsteps = std::max(nsteps, n2);
    }
    nsteps += nsteps & 1;  // the kernel runs two slots per step
    if (32 * nsteps == P) nsteps += 2;  // keep one empty slot: its c_p is exactly 0 (padding below)
    // Slots, step by step: each lane takes the next pair of its current row,
    // choosing among the row's remaining pairs the partner that adds the fewest
    // shared-memory wavefronts to its quarter-warp's partner load in this step
    // (a partner another lane already reads is free); lanes with the fewest
    // pairs left choose first.  A lane past its last row reads atom 0 as the
    // partner of its empty slots.
    std::vector<int> slots((size_t)nsteps * 32, -1);
    std::vector<int> slot_flags((size_t)nsteps * 32, 0);
    {
        std::vector<int> ri(32, 0), pi(32, 0);  // row index in the lane's list, position in the row
        std::vector<std::vector<int>> rem(32);  // remaining pairs of the current row
        for (int st = 0; st < nsteps; ++st)
            for (int qd = 0; qd < 4; ++qd) {
                WordSet<8> ph;  // partners this quarter reads in this step
                int order[8], no = 0;
                for (int l = qd * 8; l < qd * 8 + 8; ++l) {
                    if (ri[l] >= (int)lane_rows[l].size()) {
                        ph.add(0);
                        continue;
                    }
                    if (pi[l] == 0) rem[l] = rows[lane_rows[l][ri[l]]].ps;
                    order[no++] = l;
                }
                std::stable_sort(order, order + no, [&](int x, int y) { return rem[x].size() < rem[y].size(); });
                for (int t = 0; t < no; ++t) {
                    const int l = order[t];
                    const Row& r = rows[lane_rows[l][ri[l]]];
                    const int i0 = r.owner >= 0 ? r.owner : pairs[r.ps[0]].first;
                    int pick = 0, best = 1 << 30;
                    for (size_t k = 0; k < rem[l].size(); ++k) {
                        const int rk = ph.rank(pairs[rem[l][k]].first + pairs[rem[l][k]].second - i0);
                        if (rk < best) {
                            best = rk;
                            pick = (int)k;
                        }
                    }
                    const int p = rem[l][pick];
                    rem[l].erase(rem[l].begin() + pick);
                    ph.add(pairs[p].first + pairs[p].second - i0);
                    slots[(size_t)st * 32 + l] = p;
                    int fl = r.owner >= 0 ? kPairOwned : 0;
                    if (pi[l] == 0) fl |= kPairRowStart;
                    if (rem[l].empty()) {
                        fl |= kPairRowEnd;
                        ++ri[l];
                        pi[l] = 0;
                    } else {
                        ++pi[l];
                    }
                    slot_flags[(size_t)st * 32 + l] = fl;
                }
            }
    }
    // --- force-gather program: every atom's (partner, slot) entries that its
    // row does not cover go to one lane, in groups of four (the last group
    // padded with entries on an empty slot, c_p = 0, which add exactly nothing
    // whatever their partner).  Atoms are dealt longest list first to the
    // least loaded lane, preferring a quarter-warp without an atom of the same
    // index mod 8.  Group by group and position by position, each lane (fewest
    // entries left first) takes the entry that adds the fewest shared-memory
    // wavefronts to the position's partner load (its quarter-warp) and c_p
    // load (the warp); a padding entry reads a partner its quarter already
    // reads.  Entry = partner | atom << 7 | slot << 14, bit 31 on the last
    // entry of the atom's last group.  Every lane runs the same number of
    // groups (empty groups are all zero and never stored).
    int zero_slot = -1;
    for (int sl = 0; sl < (int)slots.size() && zero_slot < 0; ++sl)
        if (slots[sl] < 0) zero_slot = sl;
    if (zero_slot < 0) return ADG_EINVAL;  // unreachable: nsteps keeps one slot empty
    std::vector<std::vector<std::pair<int, int>>> inc(na);
    for (int sl = 0; sl < (int)slots.size(); ++sl) {
        const int p = slots[sl];
        if (p < 0) continue;
        const int i = pairs[p].first, j = pairs[p].second;
        if (owner[p] != i) inc[i].emplace_back(j, sl);
        if (owner[p] != j) inc[j].emplace_back(i, sl);
    }
    std::vector<int> by_deg(N);
    for (int pos = 0; pos < N; ++pos) by_deg[pos] = idx_of(pos);
    std::stable_sort(by_deg.begin(), by_deg.end(), [&](int x, int y) { return inc[x].size() > inc[y].size(); });
    std::vector<std::vector<int>> lane_atoms(32);
    std::vector<int> gload(32, 0);
    {
        std::vector<int> qres(4, 0);
        for (int i : by_deg) {
            if (inc[i].empty()) continue;
            const int m = *std::min_element(gload.begin(), gload.end());
            int lane = -1;
            for (int l = 0; l < 32 && lane < 0; ++l)
                if (gload[l] == m && !(qres[l / 8] >> (i % 8) & 1)) lane = l;
            if (lane < 0)
                for (int l = 0; l < 32 && lane < 0; ++l)
                    if (gload[l] == m) lane = l;
            lane_atoms[lane].push_back(i);
            gload[lane] += (int)(inc[i].size() + 3) / 4;
            qres[lane / 8] |= 1 << (i % 8);
        }
    }
    const int ngroups = *std::max_element(gload.begin(), gload.end());
    std::vector<uint32_t> gent((size_t)ngroups * 128, 0u);
    {
        std::vector<int> ai(32, 0), left(32, 0);           // atom index in the lane's list, groups left
        std::vector<std::vector<std::pair<int, int>>> pool(32);  // entries of the current atom not yet placed
        for (int k = 0; k < ngroups; ++k) {
            for (int l = 0; l < 32; ++l) {
                if (ai[l] >= (int)lane_atoms[l].size()) continue;
                if (left[l] == 0) {
                    const int a2 = lane_atoms[l][ai[l]];
                    pool[l] = inc[a2];
                    while (pool[l].size() % 4) pool[l].emplace_back(a2, zero_slot);
                    left[l] = (int)pool[l].size() / 4;
                }
            }
            for (int q = 0; q < 4; ++q) {
                WordSet<32> cb;    // c_p slots the warp reads at this position
                WordSet<8> ph[4];  // partners each quarter reads at this position
                int order[32], no = 0;
                for (int l = 0; l < 32; ++l) {
                    if (ai[l] >= (int)lane_atoms[l].size()) {  // an all-zero entry: slot 0, atom 0
                        cb.add(0);
                        ph[l / 8].add(0);
                        continue;
                    }
                    order[no++] = l;
                }
                std::stable_sort(order, order + no, [&](int x, int y) { return pool[x].size() < pool[y].size(); });
                for (int t = 0; t < no; ++t) {
                    const int l = order[t];
                    const int a2 = lane_atoms[l][ai[l]];
                    WordSet<8>& pq = ph[l / 8];
                    // a padding entry (empty slot, c_p = 0) adds nothing whatever its
                    // partner: it reads an atom its quarter already reads, if any
                    const int pad_partner = pq.n > 0 ? pq.words[0] : a2;
                    int pick = 0, best = 1 << 30;
                    for (size_t c = 0; c < pool[l].size(); ++c) {
                        const bool pad = pool[l][c].second == zero_slot;
                        const int pt = pad ? pad_partner : pool[l][c].first;
                        const int rk = pq.rank(pt) + cb.rank(pool[l][c].second);
                        if (rk < best) {
                            best = rk;
                            pick = (int)c;
                        }
                    }
                    std::pair<int, int> en = pool[l][pick];
                    pool[l].erase(pool[l].begin() + pick);
                    if (en.second == zero_slot) en.first = pad_partner;
                    pq.add(en.first);
                    cb.add(en.second);
                    uint32_t e = (uint32_t)en.first | ((uint32_t)a2 << 7) | ((uint32_t)en.second << 14);
                    if (q == 3 && left[l] == 1) e |= 0x80000000u;
                    gent[((size_t)k * 32 + l) * 4 + q] = e;
                }
            }
            for (int l = 0; l < 32; ++l) {
                if (ai[l] >= (int)lane_atoms[l].size()) continue;
                if (--left[l] == 0) ++ai[l];
            }
        }
    }
    if (ngroups > 0) {
        std::vector<int> blk((size_t)ngroups * 32, -1);
        for (int l = 0; l < 32; ++l) {
            int k = 0;
            for (int a2 : lane_atoms[l])
                for (int g = 0; g < (int)(inc[a2].size() + 3) / 4; ++g) blk[(size_t)k++ * 32 + l] = a2;
        }
        std::vector<char> empty_slot(slots.size(), 0);
        for (size_t sl = 0; sl < slots.size(); ++sl) empty_slot[sl] = slots[sl] < 0;
        std::vector<char> used(na, 0);
        for (int i = 0; i < na; ++i) used[i] = src_of[i] >= 0;
        GatherRefine gr(gent, ngroups, used, blk, empty_slot);
        gr.run(kGatherRefinePerEntry * (long)gent.size());
        gr.store();
    }
    // --- device header
    LigandDev h;
    memset(&h, 0, sizeof(h));
    h.natoms = N;
    h.ntors = T;
    h.npairs = P;
    h.nsteps = nsteps;
    h.gsteps = ngroups;
    double c[3] = {0, 0, 0};
    for (int i = 0; i < N; ++i)
        for (int a = 0; a < 3; ++a) c[a] += d->xyz[3 * i + a];
    h.cx = (float)(c[0] / N);
    h.cy = (float)(c[1] / N);
    h.cz = (float)(c[2] / N);
    const double B = (double)ff->ms_eps0 - ff->ms_A;
    h.e_cap = ff->e_cap;
    h.rmin2 = ff->r_min * ff->r_min;
    h.ms_A = ff->ms_A;
    h.ms_B = (float)B;
    h.ms_k = ff->ms_k;
    h.ms_lb = (float)((double)ff->ms_lambda * B);
    h.inv_2s2 = (float)(1.0 / (2.0 * (double)ff->sigma * ff->sigma));
    h.inv_s2 = (float)(1.0 / ((double)ff->sigma * ff->sigma));
    h.k_out = ff->k_out;
    h.wq = (float)((double)ff->w_elec * ff->coulomb);
    h.apl = apl;
    h.last_idx = idx_of(N - 1);
    for (int n = 0; n < N; ++n) {
        const int i = old_of[n], x = idx_of(n);
        h.ref[x] = make_float4(d->xyz[3 * i], d->xyz[3 * i + 1], d->xyz[3 * i + 2], d->charge[i]);
        h.tf[x] = d->type[i] | (fnew[frag[i]] << 8);
        h.old_of_new[x] = i;
    }
    h.nfrag = nf;
    h.maxlev = maxlev;
    for (int fi = 0; fi < nf; ++fi) {
        const int f = forder[fi];
        h.fpar[fi] = fpar[f] >= 0 ? fnew[fpar[f]] : -1;
        h.ftor[fi] = ftor[f];
        h.flev[fi] = flev[f];
    }
    for (int k = 0; k < T; ++k) {
        h.ta[k] = idx_of(nw[ta[k]]);
        h.tb[k] = idx_of(nw[tb[k]]);
        h.hi_idx[k] = idx_of(shi[k] - 1);
        h.lo_idx[k] = slo[k] > 0 ? idx_of(slo[k] - 1) : -1;
        const float* pa = d->xyz + 3 * ta[k];
        const float* pb = d->xyz + 3 * tb[k];
        double u[3] = {(double)pb[0] - pa[0], (double)pb[1] - pa[1], (double)pb[2] - pa[2]};
        const double un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        if (!(un > 0)) return ADG_ETOPO;
        h.tpt[k] = make_float4(pa[0], pa[1], pa[2], 0.f);
        h.tax[k] = make_float4((float)(u[0] / un), (float)(u[1] / un), (float)(u[2] / un), 0.f);
    }
    // --- pair records: per slot (c12, cm, cd, ij), stored for the kernel's
    // two-slot steps as pk[a] = (c12_a, c12_b, cm_a, cm_b) and
    // pk[b] = (cd_a, cd_b, ij_a, ij_b), slots a = 2t * 32 + lane and b = a + 32,
    // so each coefficient pair arrives as one two-wide operand.  Empty slots
    // (the tail of a lane's list) have zero coefficients and the uncharged pad
    // atom as their row atom, loaded at the lane's first empty slot.
    const int ns = nsteps * 32;
    const uint32_t pad_atom = (uint32_t)na;
    std::vector<uint4> rec(ns, make_uint4(0, 0, 0, 0));  // moved as bits
    for (int s = 0; s < ns; ++s) {
        const int p = slots[s];
        if (p < 0) {
            const bool first = s < 32 || slots[s - 32] >= 0;
            rec[s].w = pad_atom | (first ? (uint32_t)kPairRowStart : 0u);
            continue;
        }
        // the owner, if any, goes first: the kernel sums the force on ij & 255
        const int i = owner[p] == pairs[p].second ? pairs[p].second : pairs[p].first;
        const int j = pairs[p].first + pairs[p].second - i;
        const int ti = d->type[src_of[i]], tj = d->type[src_of[j]];
        const double qi = d->charge[src_of[i]], qj = d->charge[src_of[j]];
        float c12, c6, c10;
        pair_coefs(*ff, ti, tj, &c12, &c6, &c10);
        const bool hb = c10 != 0.f;
        const uint32_t tgt = (slot_flags[s] & kPairOwned) ? (uint32_t)i : (uint32_t)na;
        const int ij = (int)((uint32_t)(i | (j << 16) | slot_flags[s] | (hb ? kPairHB : 0)) | (tgt << 24));
        const float cd = (float)((double)ff->w_desolv * (((double)ff->solpar[ti] + (double)ff->qasp * fabs(qi)) * ff->vol[tj] +
                                                         ((double)ff->solpar[tj] + (double)ff->qasp * fabs(qj)) * ff->vol[ti]));
        const float cm = hb ? c10 : c6;
        uint4& r = rec[s];
        memcpy(&r.x, &c12, 4);
        memcpy(&r.y, &cm, 4);
        memcpy(&r.z, &cd, 4);
        memcpy(&r.w, &ij, 4);
    }
    std::vector<uint4> pk(ns);
    for (int a = 0; a < ns; a += 64)
        for (int l = 0; l < 32; ++l) {
            const uint4 ra = rec[a + l], rb = rec[a + 32 + l];
            pk[a + l] = make_uint4(ra.x, rb.x, ra.y, rb.y);
            pk[a + 32 + l] = make_uint4(ra.z, rb.z, ra.w, rb.w);
        }
    const size_t off_pk = align_up(sizeof(LigandDev), 256);
    const size_t off_gent = align_up(off_pk + sizeof(uint4) * ns, 256);
    const size_t bytes = align_up(off_gent + sizeof(uint32_t) * gent.size(), 256);
    h.blob_bytes = (int)bytes;
    h.off_pk = (int)off_pk;
    h.off_gent = (int)off_gent;
    pl.h = h;
    pl.pk = std::move(pk);
    pl.gent = std::move(gent);
    pl.nf = nf;
    pl.sum_moving = 0;
    for (int k = 0; k < T; ++k) pl.sum_moving += shi[k] - slo[k];
    return ADG_OK;
}

// Shared-memory wavefronts of one warp access, from the word each lane
// touches (-1: lane inactive); lanes on the same word share it.  A 16-byte
// access runs as four quarter-warp phases, each taking as many wavefronts as
// the most distinct words on one of its eight 16-byte bank groups; a 4-byte
// access takes as many as the most distinct words on one of the 32 banks.
// `ideal` adds what the access would take without bank conflicts.
int wavefronts(const int* w, bool wide, int* ideal)
{
    int tot = 0, best = 0;
    const int nphase = wide ? 4 : 1, lanes = wide ? 8 : 32, banks = wide ? 8 : 32;
    for (int ph = 0; ph < nphase; ++ph) {
        int cnt[32] = {0}, any = 0, m = 0;
        for (int l = ph * lanes; l < (ph + 1) * lanes; ++l) {
            if (w[l] < 0) continue;
            bool dup = false;
            for (int k = ph * lanes; k < l && !dup; ++k) dup = w[k] == w[l];
            if (dup) continue;
            any = 1;
            m = std::max(m, ++cnt[w[l] % banks]);
        }
        tot += m;
        best += any;
    }
    *ideal += best;
    return tot;
}

// The scoring kernel's shared-memory accesses in the pair loop and the force
// gather of one energy+gradient evaluation, walked over the plan.
void model_schedule(const LigandPlan& pl, adg_schedule_stats* out)
{
    const LigandDev& h = pl.h;
    int w[32], pi = 0, gi = 0;
    int pw = 0, gw = 0;
    const int ns = h.nsteps * 32;
    for (int a0 = 0; a0 < ns; a0 += 64) {
        uint32_t ij[2][32];
        for (int l = 0; l < 32; ++l) {
            ij[0][l] = pl.pk[a0 + 32 + l].z;
            ij[1][l] = pl.pk[a0 + 32 + l].w;
        }
        for (int r = 0; r < 2; ++r) {  // the two record loads: consecutive words
            for (int l = 0; l < 32; ++l) w[l] = a0 + 32 * r + l;
            pw += wavefronts(w, true, &pi);
        }
        for (int sl = 0; sl < 2; ++sl) {
            for (int l = 0; l < 32; ++l) w[l] = (ij[sl][l] & kPairRowStart) ? (int)(ij[sl][l] & 255) : -1;
            pw += wavefronts(w, true, &pi);  // row atom at the row's first slot
            for (int l = 0; l < 32; ++l) w[l] = (int)((ij[sl][l] >> 16) & 127);
            pw += wavefronts(w, true, &pi);  // partner
        }
        for (int sl = 0; sl < 2; ++sl) {  // c_p stores: consecutive
            for (int l = 0; l < 32; ++l) w[l] = a0 + 32 * sl + l;
            pw += wavefronts(w, false, &pi);
        }
        for (int sl = 0; sl < 2; ++sl) {  // row-end force stores
            for (int l = 0; l < 32; ++l) w[l] = (ij[sl][l] & kPairRowEnd) ? (int)(ij[sl][l] >> 24) : -1;
            pw += wavefronts(w, true, &pi);
        }
    }
    for (int k = 0; k < h.gsteps; ++k) {
        const uint32_t* e = pl.gent.data() + (size_t)k * 128;
        for (int l = 0; l < 32; ++l) w[l] = k * 32 + l;
        gw += wavefronts(w, true, &gi);  // the group's four entries
        for (int q = 0; q < 4; ++q) {
            for (int l = 0; l < 32; ++l) w[l] = (int)((e[l * 4 + q] >> 14) & 0xffff);
            gw += wavefronts(w, false, &gi);  // c_p
        }
        for (int q = 0; q < 4; ++q) {
            for (int l = 0; l < 32; ++l) w[l] = (int)(e[l * 4 + q] & 127);
            gw += wavefronts(w, true, &gi);  // partner coordinates
        }
        // flush at the atom's last group: its two sums written
        for (int l = 0; l < 32; ++l) w[l] = (e[l * 4 + 3] >> 31) ? (int)((e[l * 4] >> 7) & 127) : -1;
        gw += wavefronts(w, true, &gi);
    }
    out->pair_wavefronts = pw;
    out->pair_wavefronts_ideal = pi;
    out->gather_wavefronts = gw;
    out->gather_wavefronts_ideal = gi;
}

}  // namespace

extern "C" {

int adg_ligand_schedule(const adg_forcefield* ff, const adg_ligand_desc* d, adg_schedule_stats* out)
{
    if (!ff || !d || !out) return ADG_EINVAL;
    LigandPlan pl;
    const int rc = plan_ligand(ff, d, pl);
    if (rc != ADG_OK) return rc;
    memset(out, 0, sizeof(*out));
    out->natoms = pl.h.natoms;
    out->npairs = pl.h.npairs;
    out->nsteps = pl.h.nsteps;
    out->gsteps = pl.h.gsteps;
    out->empty_slots = pl.h.nsteps * 32 - pl.h.npairs;
    model_schedule(pl, out);
    return ADG_OK;
}

int adg_ligand_create(adg_ctx* ctx, const adg_forcefield* ff, const adg_ligand_desc* d, adg_ligand** out)
{
    if (!ctx || !ff || !d || !out) return ADG_EINVAL;
    *out = nullptr;
    LigandPlan pl;
    const int rc = plan_ligand(ff, d, pl);
    if (rc != ADG_OK) return rc;
    const LigandDev& h = pl.h;
    const int N = h.natoms, T = h.ntors, P = h.npairs, nf = pl.nf;
    const size_t bytes = (size_t)h.blob_bytes, off_pk = (size_t)h.off_pk, off_gent = (size_t)h.off_gent;
    const int ns = (int)pl.pk.size();
    CK(ctx, cudaSetDevice(ctx->device));
    adg_ligand* L = new (std::nothrow) adg_ligand();
    if (!L) return ADG_ENOMEM;
    std::vector<char> host(bytes, 0);
    memcpy(host.data(), &h, sizeof(h));
    memcpy(host.data() + off_pk, pl.pk.data(), sizeof(uint4) * ns);
    memcpy(host.data() + off_gent, pl.gent.data(), sizeof(uint32_t) * pl.gent.size());
    cudaError_t e = cudaMalloc(&L->blob, bytes);
    if (e == cudaSuccess) e = cudaMemcpyAsync(L->blob, host.data(), bytes, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        if (L->blob) cudaFree(L->blob);
        delete L;
        return cuda_fail(ctx, e, "ligand upload");
    }
    char* base = (char*)L->blob;
    L->ctx = ctx;
    L->device = ctx->device;
    L->ref.hdr = (const LigandDev*)base;
    L->ref.pairs.pk = (const float4*)(base + off_pk);
    L->ref.pairs.gent = (const uint32_t*)(base + off_gent);
    L->nslots = ns;
    L->natoms = N;
    L->ntors = T;
    L->npairs = P;
    L->apl = apl_for(N);
    L->bytes = bytes;
    L->sum_moving = pl.sum_moving;
    // descriptors of the ligand for the triage network (see adg_ligand_descriptors)
    {
        float* D = L->desc;
        for (int q = 0; q < ADG_NDESC; ++q) D[q] = 0.f;
        D[0] = (float)N;
        D[1] = (float)T;
        D[2] = (float)P;
        double cx = 0, cy = 0, cz = 0, sq = 0, sq2 = 0;
        for (int i = 0; i < N; ++i) {
            D[3 + d->type[i]] += 1.f;
            cx += d->xyz[3 * i];
            cy += d->xyz[3 * i + 1];
            cz += d->xyz[3 * i + 2];
            sq += fabs((double)d->charge[i]);
            sq2 += (double)d->charge[i] * d->charge[i];
        }
        cx /= N;
        cy /= N;
        cz /= N;
        double rg = 0, rmax = 0;
        for (int i = 0; i < N; ++i) {
            const double dx = d->xyz[3 * i] - cx, dy = d->xyz[3 * i + 1] - cy, dz = d->xyz[3 * i + 2] - cz;
            const double r2 = dx * dx + dy * dy + dz * dz;
            rg += r2;
            rmax = std::max(rmax, sqrt(r2));
        }
        D[10] = (float)sq;
        D[11] = (float)sq2;
        D[12] = (float)sqrt(rg / N);
        D[13] = (float)rmax;
        D[14] = (float)nf;
        D[15] = T > 0 ? (float)L->sum_moving / (float)T : 0.f;
    }
    ctx->stats.h2d_bytes += (int64_t)bytes;
    *out = L;
    return ADG_OK;
}

int adg_ligand_set_stream_id(adg_ligand* lig, int64_t id)
{
    if (!lig || id < -1 || id > (int64_t)0xffffffffu) return ADG_EINVAL;
    lig->stream_id = id;
    return ADG_OK;
}

int adg_ligand_descriptors(const adg_ligand* lig, float* out)
{
    if (!lig || !out) return ADG_EINVAL;
    for (int q = 0; q < ADG_NDESC; ++q) out[q] = lig->desc[q];
    return ADG_OK;
}

int adg_ligand_destroy(adg_ligand* lig)
{
    if (!lig) return ADG_EINVAL;
    cudaSetDevice(lig->device);
    cudaFree(lig->blob);
    delete lig;
    return ADG_OK;
}

int adg_ligand_info(const adg_ligand* lig, adg_ligand_stats* out)
{
    if (!lig || !out) return ADG_EINVAL;
    out->natoms = lig->natoms;
    out->ntors = lig->ntors;
    out->npairs = lig->npairs;
    out->sum_moving = lig->sum_moving;
    out->device_bytes = (int64_t)lig->bytes;
    return ADG_OK;
}

int adg_score(adg_ctx* ctx, const adg_receptor* rec, const adg_ligand* lig, const float* genes, int npose,
              float* energy, float* grad, int grad_kind)
{
    if (!ctx || !rec || !lig || npose < 0 || (npose > 0 && (!genes || !energy))) return ADG_EINVAL;
    if (grad_kind != ADG_GRAD_NONE && grad_kind != ADG_GRAD_GENES && grad_kind != ADG_GRAD_TANGENT) return ADG_EINVAL;
    if (grad_kind != ADG_GRAD_NONE && npose > 0 && !grad) return ADG_EINVAL;
    if (npose == 0) return ADG_OK;
    CK(ctx, cudaSetDevice(ctx->device));
    CK(ctx, launch_score(ctx->stream, rec->maps, lig->ref, make_geo(lig->apl, lig->nslots, lig->bytes), genes, npose, energy, grad,
                         grad_kind));
    ctx->stats.kernel_launches += 1;
    return ADG_OK;
}

int adg_score_multi(adg_ctx* ctx, const adg_receptor* rec, const adg_ligand* const* ligs, int nlig, const int* npose,
                    const float* genes, float* energy, float* grad, int grad_kind)
{
    if (!ctx || !rec || !ligs || nlig < 0 || (nlig > 0 && !npose)) return ADG_EINVAL;
    if (grad_kind != ADG_GRAD_NONE && grad_kind != ADG_GRAD_GENES && grad_kind != ADG_GRAD_TANGENT) return ADG_EINVAL;
    long total = 0;
    for (int i = 0; i < nlig; ++i) {
        if (!ligs[i] || ligs[i]->ctx != ctx || npose[i] < 0) return ADG_EINVAL;
        total += npose[i];
    }
    if (total > 0 && (!genes || !energy || (grad_kind != ADG_GRAD_NONE && !grad))) return ADG_EINVAL;
    if (total == 0) return ADG_OK;
    if (total > (1l << 30)) return ADG_ETOOBIG;
    CK(ctx, cudaSetDevice(ctx->device));
    // one launch per atoms-per-lane width, the widths on concurrent streams;
    // rows keep the caller's ligand order
    std::vector<long> row0(nlig);
    for (int i = 0, r = 0; i < nlig; ++i) {
        row0[i] = r;
        r += npose[i];
    }
    int nsm = 148;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device);
    struct Width {
        Geo g;
        int nblocks;
        size_t o_ref, o_bl, o_b0, o_r0, o_np, o_nb;
    };
    std::vector<Width> widths;
    std::vector<char> host;  // every width's tables, in one buffer
    auto put = [&](const void* src, size_t n) {
        const size_t o = align_up(host.size(), 256);
        host.resize(o + n);
        if (n) memcpy(host.data() + o, src, n);
        return o;
    };
    for (int apl = 1; apl <= 4; ++apl) {
        std::vector<int> members;
        int nslots = 32;
        size_t lig_bytes = 0;
        for (int i = 0; i < nlig; ++i)
            if (ligs[i]->apl == apl && npose[i] > 0) {
                members.push_back(i);
                nslots = std::max(nslots, ligs[i]->nslots);
                lig_bytes = std::max(lig_bytes, ligs[i]->bytes);
            }
        if (members.empty()) continue;
        Width w;
        w.g = make_geo(apl, nslots, lig_bytes);
        const int nm = (int)members.size();
        // poses per warp: up to 8, while the launch keeps at least two waves of blocks
        long width_poses = 0;
        for (int m = 0; m < nm; ++m) width_poses += npose[members[m]];
        const long waves2 = 2l * nsm * 2 * w.g.wpb;  // warps in two waves of two blocks per SM
        const int ppw = (int)std::max(1l, std::min(8l, width_poses / std::max(1l, waves2)));
        std::vector<LigandRef> refs(nm);
        std::vector<int> blk0(nm), rows(nm), np(nm), nblk(nm), blk_lig;
        for (int m = 0; m < nm; ++m) {
            const int i = members[m];
            refs[m] = ligs[i]->ref;
            blk0[m] = (int)blk_lig.size();
            rows[m] = (int)row0[i];
            np[m] = npose[i];
            const int nb = (npose[i] + w.g.wpb * ppw - 1) / (w.g.wpb * ppw);
            nblk[m] = nb;
            for (int b = 0; b < nb; ++b) blk_lig.push_back(m);
        }
        w.nblocks = (int)blk_lig.size();
        w.o_ref = put(refs.data(), sizeof(LigandRef) * nm);
        w.o_bl = put(blk_lig.data(), sizeof(int) * blk_lig.size());
        w.o_b0 = put(blk0.data(), sizeof(int) * nm);
        w.o_r0 = put(rows.data(), sizeof(int) * nm);
        w.o_np = put(np.data(), sizeof(int) * nm);
        w.o_nb = put(nblk.data(), sizeof(int) * nm);
        widths.push_back(w);
    }
    cudaStream_t st = ctx->stream;
    // the tables are uploaded only when they differ from the last call's: the
    // buffer is rewritten in stream order, after every earlier launch that
    // read it (earlier calls joined their streams back into this one)
    if (host != ctx->multi_host) {
        if (host.size() > ctx->multi_cap) {
            if (ctx->multi_dev) CK(ctx, cudaFreeAsync(ctx->multi_dev, st));
            ctx->multi_dev = nullptr;
            ctx->multi_cap = 0;
            CK(ctx, cudaMallocAsync(&ctx->multi_dev, host.size(), st));
            ctx->multi_cap = host.size();
        }
        ctx->multi_host.clear();  // stale until the copy below is issued
        CK(ctx, cudaMemcpyAsync(ctx->multi_dev, host.data(), host.size(), cudaMemcpyHostToDevice, st));
        ctx->multi_host = host;
        ctx->stats.h2d_bytes += (int64_t)host.size();
    }
    while (ctx->class_streams.size() + 1 < widths.size()) {
        cudaStream_t s2;
        CK(ctx, cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
        ctx->class_streams.push_back(s2);
    }
    cudaEvent_t fork = nullptr;
    if (widths.size() > 1) {
        CK(ctx, take_event(ctx, &fork));
        CK(ctx, cudaEventRecord(fork, st));
    }
    const char* dev = (const char*)ctx->multi_dev;
    cudaError_t e = cudaSuccess;
    for (size_t k = 0; k < widths.size() && e == cudaSuccess; ++k) {
        const Width& w = widths[k];
        cudaStream_t sk = k == 0 ? st : ctx->class_streams[k - 1];
        if (k > 0) e = cudaStreamWaitEvent(sk, fork, 0);
        if (e != cudaSuccess) break;
        ScoreMultiDev J;
        J.ligs = (const LigandRef*)(dev + w.o_ref);
        J.blk_lig = (const int*)(dev + w.o_bl);
        J.lig_blk0 = (const int*)(dev + w.o_b0);
        J.lig_row0 = (const int*)(dev + w.o_r0);
        J.lig_npose = (const int*)(dev + w.o_np);
        J.lig_nblk = (const int*)(dev + w.o_nb);
        J.stride = ADG_MAX_GENES;
        e = launch_score_multi(sk, rec->maps, J, w.nblocks, w.g, genes, energy,
                               grad_kind == ADG_GRAD_NONE ? nullptr : grad, grad_kind);
        ctx->stats.kernel_launches += 1;
    }
    // join: the context's stream waits for every width
    for (size_t k = 1; k < widths.size(); ++k) {
        cudaEvent_t done;
        const cudaError_t e1 = take_event(ctx, &done);
        if (e1 != cudaSuccess) return cuda_fail(ctx, e1, "adg_score_multi");
        cudaEventRecord(done, ctx->class_streams[k - 1]);
        cudaStreamWaitEvent(st, done, 0);
        ctx->ev_free.push_back(done);
    }
    if (fork) ctx->ev_free.push_back(fork);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "adg_score_multi");
    return ADG_OK;
}

int adg_pose(adg_ctx* ctx, const adg_ligand* lig, const float* genes, int npose, float* xyz)
{
    if (!ctx || !lig || npose < 0 || (npose > 0 && (!genes || !xyz))) return ADG_EINVAL;
    if (npose == 0) return ADG_OK;
    CK(ctx, cudaSetDevice(ctx->device));
    CK(ctx, launch_pose(ctx->stream, lig->ref, make_geo(lig->apl, lig->nslots, lig->bytes), genes, npose, xyz));
    ctx->stats.kernel_launches += 1;
    return ADG_OK;
}

int adg_philox(adg_ctx* ctx, const uint32_t* ctr, int n, uint64_t key, uint32_t* out)
{
    if (!ctx || n < 0 || (n > 0 && (!ctr || !out))) return ADG_EINVAL;
    if (((uintptr_t)ctr | (uintptr_t)out) & 15u) return ADG_EINVAL;  // read and written as uint4
    if (n == 0) return ADG_OK;
    CK(ctx, cudaSetDevice(ctx->device));
    CK(ctx, launch_philox(ctx->stream, ctr, n, (uint32_t)(key & 0xffffffffu), (uint32_t)(key >> 32), out));
    ctx->stats.kernel_launches += 1;
    return ADG_OK;
}

namespace {

// One shape class of a dock call: the ligands sharing an atoms-per-lane
// width, docked by one graph on one stream.
struct ClassRun {
    std::vector<int> ligs;   // indices into the call's ligand list
    Geo geo;
    DockDev D;
    int* d_active = nullptr;
    int* d_gen = nullptr;
    ResultDev* d_res = nullptr;
    cudaStream_t stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;  // around the generation loop (timing mode)
    SearchDev S;   // the call's search parameters, nrun = this group's runs per ligand
    int run0 = 0;  // the group's first run
};

// A single ligand's runs go out in this many concurrent groups (see dock_impl).
constexpr int kRunParts = 2;

void fill_search(const adg_search_params* p, SearchDev& S)
{
    S.nrun = p->nrun;
    S.pop = p->pop_size;
    S.nev = p->nev;
    S.max_gen = p->max_gen;
    S.ls_method = p->ls_method;
    S.ls_max_iters = p->ls_max_iters;
    S.elitism = p->elitism;
    S.thr_ls = prob_threshold(p->ls_rate);
    S.thr_cross = prob_threshold(p->crossover_rate);
    S.thr_mut = prob_threshold(p->mutation_rate);
    S.thr_tour = prob_threshold(p->tournament_rate);
    S.sw_rho0 = p->sw_rho0;
    S.sw_rho_min = p->sw_rho_min;
    S.sw_expand = p->sw_expand;
    S.sw_contract = p->sw_contract;
    S.sw_succ = p->sw_succ;
    S.sw_fail = p->sw_fail;
    S.sw_scale_t = p->sw_scale_t;
    S.sw_scale_rot = p->sw_scale_rot;
    S.sw_scale_tors = p->sw_scale_tors;
    S.ad_rho = p->ad_rho;
    S.ad_eps = p->ad_eps;
    S.mut_t = p->mut_t;
    S.mut_rot = p->mut_rot;
    S.mut_tors = p->mut_tors;
    S.key0 = (uint32_t)(p->seed & 0xffffffffu);
    S.key1 = (uint32_t)(p->seed >> 32);
    S.autostop = p->autostop != 0;
    S.stopstd = p->stopstd;
}

// ---- launch geometry of adg_dock
// Shape bucket of a ligand: atoms per lane, local-search kind, pair slots
// rounded up to 256 and blob bytes rounded up to 8 KiB.
uint32_t bucket_key(int apl, int ls, int nslots, size_t bytes, int* ns_b, int* by_b)
{
    *ns_b = (int)align_up((size_t)std::max(nslots, 1), 256);
    *by_b = (int)align_up(std::max(bytes, (size_t)1), 8192);
    return (uint32_t)apl | ((uint32_t)ls << 3) | ((uint32_t)(*ns_b / 256) << 8) | ((uint32_t)(*by_b / 8192) << 18);
}

// Time the candidate geometries (ligand staged, ligand read through L1; each
// with the block size that keeps the most warps resident) on probe poses of
// `lig`, the first member met of its bucket, and record the faster form.
int tune_shape(adg_ctx* ctx, const adg_receptor* rec, const adg_ligand* lig, int ls, int ns_b, int by_b,
               adg_tuned_shape* out)
{
    Geo cand[2];
    const int n = geo_candidates(lig->apl, lig->nslots, lig->bytes, ls, cand, 2);
    adg_tuned_shape t{};
    t.apl = lig->apl;
    t.ls_method = ls;
    t.nslots_max = ns_b;
    t.bytes_max = by_b;
    t.ncand = n;
    if (n == 0) {  // no candidate launches: keep the fixed rule
        const Geo g = make_geo(lig->apl, lig->nslots, lig->bytes);
        t.staged = g.lig_bytes > 0;
        t.warps_per_block = g.wpb;
        t.blocks_per_sm = geo_blocks_per_sm(g, ls);
        *out = t;
        return ADG_OK;
    }
    int pick = 0;
    if (n > 1) {
        int nsm = 0, smem_sm = 0, reserve = 0, optin = 0;
        CK(ctx, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
        CK(ctx, cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ctx->device));
        CK(ctx, cudaDeviceGetAttribute(&reserve, cudaDevAttrReservedSharedMemoryPerBlock, ctx->device));
        CK(ctx, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
        int bps[2], maxres = 0;
        for (int k = 0; k < n; ++k) {
            bps[k] = geo_blocks_per_sm(cand[k], ls);
            maxres = std::max(maxres, bps[k] * cand[k].wpb);
        }
        const int reps = 8, G = 7 + lig->ntors;
        const long npose = (long)nsm * maxres * 2;  // two waves of the most resident candidate
        const size_t need = align_up(sizeof(float) * npose * G, 256) + sizeof(float) * npose;
        if (need > ctx->tune_bytes) {
            CK(ctx, cudaStreamSynchronize(ctx->stream));
            if (ctx->tune_buf) cudaFree(ctx->tune_buf);
            ctx->tune_buf = nullptr;
            ctx->tune_bytes = 0;
            cudaError_t e = cudaMalloc(&ctx->tune_buf, need);
            if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? ADG_ENOMEM : cuda_fail(ctx, e, "tune buffer");
            ctx->tune_bytes = need;
        }
        float* genes = (float*)ctx->tune_buf;
        float* energy = (float*)((char*)ctx->tune_buf + align_up(sizeof(float) * npose * G, 256));
        cudaStream_t st = ctx->stream;
        const bool grad = ls == ADG_LS_ADADELTA;
        CK(ctx, launch_probe_genes(st, rec->maps, lig->ntors, (int)npose, 3.0f, 0x5eedu, genes));
        cudaEvent_t a, b;
        CK(ctx, take_event(ctx, &a));
        CK(ctx, take_event(ctx, &b));
        float best_ms[2] = {0.f, 0.f};
        for (int k = 0; k < n; ++k) {
            Geo g = cand[k];
            // pad the probe's shared memory so that it keeps the generation
            // kernel's residency whatever its own register count
            size_t pad = (size_t)(smem_sm / std::max(bps[k], 1) - reserve);
            pad = std::min(pad, (size_t)optin);
            if (pad > g.smem) g.smem = pad;
            CK(ctx, launch_tune(st, rec->maps, lig->ref, g, genes, (int)npose, reps, grad, energy));
            float best = 1e30f;
            for (int r = 0; r < 3; ++r) {
                CK(ctx, cudaEventRecord(a, st));
                CK(ctx, launch_tune(st, rec->maps, lig->ref, g, genes, (int)npose, reps, grad, energy));
                CK(ctx, cudaEventRecord(b, st));
                CK(ctx, cudaEventSynchronize(b));
                float ms = 0.f;
                CK(ctx, cudaEventElapsedTime(&ms, a, b));
                best = std::min(best, ms);
            }
            best_ms[k] = best;
            t.us_per_eval[cand[k].lig_bytes > 0 ? 0 : 1] = best * 1000.f / (float)(npose * reps);
        }
        ctx->ev_free.push_back(a);
        ctx->ev_free.push_back(b);
        ctx->stats.tune_launches += 1 + 4 * n;
        ctx->stats.kernel_launches += 1 + 4 * n;
        pick = best_ms[1] < best_ms[0] ? 1 : 0;
    }
    t.staged = cand[pick].lig_bytes > 0;
    t.warps_per_block = cand[pick].wpb;
    t.blocks_per_sm = geo_blocks_per_sm(cand[pick], ls);
    *out = t;
    return ADG_OK;
}

// Group the ligands of a dock call.  Heuristic mode: by atoms per lane with
// the fixed rule.  Tuned mode: every ligand takes the form (staged or read
// through L1) its bucket was tuned to; ligands of one width and form, in
// increasing footprint, share a group while the group's largest footprint
// keeps at least 3/4 of the warps resident that its smallest member alone
// would (fewer, larger groups leave fewer partly filled waves).
int group_ligands(adg_ctx* ctx, const adg_receptor* rec, const adg_ligand* const* ligs, int nlig, int ls,
                  std::vector<ClassRun>& cls)
{
    cls.clear();
    if (ctx->geo_mode == ADG_GEO_HEURISTIC) {
        for (int apl = 1; apl <= 4; ++apl) {
            ClassRun c;
            int nslots = 32;
            size_t lig_bytes = 0;
            for (int i = 0; i < nlig; ++i)
                if (ligs[i]->apl == apl) {
                    c.ligs.push_back(i);
                    nslots = std::max(nslots, ligs[i]->nslots);
                    lig_bytes = std::max(lig_bytes, ligs[i]->bytes);
                }
            if (c.ligs.empty()) continue;
            c.geo = make_geo(apl, nslots, lig_bytes);
            cls.push_back(c);
        }
        return ADG_OK;
    }
    std::map<int, std::vector<int>> by_form;  // apl * 2 + staged -> ligands
    for (int i = 0; i < nlig; ++i) {
        int ns_b, by_b;
        const uint32_t key = bucket_key(ligs[i]->apl, ls, ligs[i]->nslots, ligs[i]->bytes, &ns_b, &by_b);
        auto it = ctx->tuned.find(key);
        if (it == ctx->tuned.end()) {
            adg_tuned_shape t;
            const int rc = tune_shape(ctx, rec, ligs[i], ls, ns_b, by_b, &t);
            if (rc != ADG_OK) return rc;
            it = ctx->tuned.emplace(key, t).first;
        }
        by_form[ligs[i]->apl * 2 + (it->second.staged ? 1 : 0)].push_back(i);
    }
    for (auto& kv : by_form) {
        const int apl = kv.first / 2;
        const bool staged = (kv.first & 1) != 0;
        std::vector<int>& members = kv.second;
        std::sort(members.begin(), members.end(), [&](int a, int b) {
            const size_t fa = (staged ? ligs[a]->bytes : 0) + 4u * ligs[a]->nslots;
            const size_t fb = (staged ? ligs[b]->bytes : 0) + 4u * ligs[b]->nslots;
            return fa < fb;
        });
        ClassRun c;
        int nslots = 0, res_first = 0;
        size_t lig_bytes = 0;
        for (int i : members) {
            const int ns2 = std::max(nslots, ligs[i]->nslots);
            const size_t lb2 = std::max(lig_bytes, ligs[i]->bytes);
            Geo g2;
            const int res2 = geo_best(apl, ns2, staged ? lb2 : 0, staged, ls, &g2);
            if (!c.ligs.empty() && 4 * res2 < 3 * res_first) {  // close the group, start the next with ligand i
                cls.push_back(c);
                c = ClassRun();
                res_first = geo_best(apl, ligs[i]->nslots, staged ? ligs[i]->bytes : 0, staged, ls, &c.geo);
                nslots = ligs[i]->nslots;
                lig_bytes = ligs[i]->bytes;
            } else {
                if (c.ligs.empty()) res_first = res2;
                c.geo = g2;
                nslots = ns2;
                lig_bytes = lb2;
            }
            if (res_first == 0) c.geo = make_geo(apl, nslots, lig_bytes);  // nothing fits: the fixed rule's fallback
            c.ligs.push_back(i);
        }
        cls.push_back(c);
    }
    // the group with the most work goes first (on the context's stream)
    std::stable_sort(cls.begin(), cls.end(), [](const ClassRun& a, const ClassRun& b) {
        return a.ligs.size() * a.geo.na > b.ligs.size() * b.geo.na;
    });
    return ADG_OK;
}

// Build the graph of one class: prologue (clear counters, initial
// population) -> WHILE (generation, bookkeeping, loop control) -> final
// poses.  The loop runs on the device until no run of the class is active.
cudaError_t build_class_graph(adg_ctx* ctx, ClassRun& c, const MapsDev& M, const SearchDev& S, bool need_loop,
                              bool timing, int nruns)
{
    cudaStream_t cs = c.stream;
    cudaGraph_t pro = nullptr, epi = nullptr, g = nullptr;
    cudaError_t e;
    // prologue
    if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed)) != cudaSuccess) return e;
    cudaMemsetAsync(c.D.evals, 0, sizeof(unsigned long long) * 2 * nruns, cs);
    cudaMemsetAsync(c.D.gen_done, 0, sizeof(int) * nruns, cs);
    cudaMemsetAsync(c.D.stopped, 0, sizeof(int) * nruns, cs);
    if (c.D.best_trace)  // all-ones words: NaN until a generation writes the entry
        cudaMemsetAsync(c.D.best_trace, 0xff, sizeof(float) * nruns * c.D.best_trace_len, cs);
    cudaMemsetAsync(c.d_active, 0, sizeof(int), cs);
    cudaMemsetAsync(c.d_gen, 0, sizeof(int), cs);  // generations completed by the loop
    launch_dock_init(cs, M, S, c.D, c.geo);
    e = cudaStreamEndCapture(cs, &pro);
    if (e != cudaSuccess) return e;
    // epilogue
    if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed)) != cudaSuccess) return e;
    launch_dock_finalize(cs, M, S, c.D, c.geo, c.d_res);
    if ((e = cudaStreamEndCapture(cs, &epi)) != cudaSuccess) return e;
    // assemble
    if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) return e;
    cudaGraphNode_t n_pro, n_epi, n_t0 = nullptr, n_t1 = nullptr, n_loop = nullptr;
    if ((e = cudaGraphAddChildGraphNode(&n_pro, g, nullptr, 0, pro)) != cudaSuccess) return e;
    cudaGraphNode_t last = n_pro;
    if (timing) {
        if ((e = cudaGraphAddEventRecordNode(&n_t0, g, &last, 1, c.t0)) != cudaSuccess) return e;
        last = n_t0;
    }
    if (need_loop) {
        cudaGraphConditionalHandle h;
        if ((e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault)) != cudaSuccess) return e;
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        if ((e = cudaGraphAddNode(&n_loop, g, &last, nullptr, 1, &np)) != cudaSuccess) return e;
        cudaGraph_t body = np.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) return e;
        launch_dock_generation(cs, M, S, c.D, c.geo, 0, c.d_gen);
        launch_dock_count_active(cs, S, c.D, 0, c.d_active, c.d_gen);
        launch_dock_loop_ctl(cs, h, c.d_gen, c.d_active);
        if ((e = cudaStreamEndCapture(cs, &body)) != cudaSuccess) return e;
        last = n_loop;
    }
    if (timing) {
        if ((e = cudaGraphAddEventRecordNode(&n_t1, g, &last, 1, c.t1)) != cudaSuccess) return e;
        last = n_t1;
    }
    if ((e = cudaGraphAddChildGraphNode(&n_epi, g, &last, 1, epi)) != cudaSuccess) return e;
    e = cudaGraphInstantiate(&c.exec, g, 0);
    cudaGraphDestroy(pro);
    cudaGraphDestroy(epi);
    cudaGraphDestroy(g);
    return e;
}

}  // namespace

namespace {

int dock_impl(adg_ctx* ctx, const adg_receptor* rec, const adg_ligand* const* ligs, int nlig,
              const adg_search_params* p, adg_result* out, adg_dock_trace* trace, float* best_trace, int ntrace)
{
    if (!ctx || !rec || !ligs || nlig <= 0 || !p || !out) return ADG_EINVAL;
    if (ntrace < 0 || (ntrace > 0 && !best_trace)) return ADG_EINVAL;
    if (p->nrun <= 0 || p->nrun > 65535 || p->pop_size < 2 || p->pop_size > 65535 || p->nev < 0 || p->max_gen < 0 ||
        p->ls_max_iters < 0 || p->elitism < 0 || p->elitism > 1 || p->ls_method < 0 || p->ls_method > 2)
        return ADG_EINVAL;
    if (trace && (nlig != 1 || trace->ngen < 0)) return ADG_EINVAL;
    for (int i = 0; i < nlig; ++i)
        if (!ligs[i] || ligs[i]->ctx != ctx) return ADG_EINVAL;
    CK(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    // --- ligand groups, one graph each
    std::vector<ClassRun> cls;
    int rc = group_ligands(ctx, rec, ligs, nlig, p->ls_method, cls);
    if (rc != ADG_OK) return rc;
    SearchDev S;
    fill_search(p, S);
    for (ClassRun& c : cls) c.S = S;
    // One ligand's runs in two halves on two concurrent graphs: the last,
    // partly filled wave of one half's generation launch overlaps the other
    // half's next generation.  Runs are independent and their random streams
    // are keyed by the run index, so the results do not change.
    if (!trace && cls.size() == 1 && cls[0].ligs.size() == 1 && p->nrun >= 4 * kRunParts) {
        const int lig0 = cls[0].ligs[0];
        const Geo geo0 = cls[0].geo;
        cls.resize(kRunParts);
        for (int q = 0, r0 = 0; q < kRunParts; ++q) {
            cls[q].ligs.assign(1, lig0);
            cls[q].geo = geo0;
            cls[q].S = S;
            cls[q].run0 = r0;
            cls[q].S.nrun = (p->nrun + kRunParts - 1 - q) / kRunParts;
            r0 += cls[q].S.nrun;
        }
    }
    ctx->stats.dock_groups += (int64_t)cls.size();
    const int tr_ngen = trace ? trace->ngen : 0;
    const long tr_slots = trace ? (long)p->nrun * tr_ngen * p->pop_size : 0;
    // --- arena layout, class after class
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    struct Offs {
        size_t g0, g1, e0, e1, ev, gd, hist, stop, act, gen, lr, id, res, bt;
    };
    std::vector<Offs> offs(cls.size());
    for (size_t k = 0; k < cls.size(); ++k) {
        const long nruns = (long)cls[k].ligs.size() * cls[k].S.nrun, nind = nruns * p->pop_size;
        Offs& o = offs[k];
        o.g0 = take(sizeof(float) * nind * kGeneStride);
        o.g1 = take(sizeof(float) * nind * kGeneStride);
        o.e0 = take(sizeof(float) * nind);
        o.e1 = take(sizeof(float) * nind);
        o.ev = take(sizeof(unsigned long long) * 2 * nruns);
        o.gd = take(sizeof(int) * nruns);
        o.hist = take(sizeof(float) * 10 * nruns);
        o.stop = take(sizeof(int) * nruns);
        o.act = take(sizeof(int) * 2);
        o.gen = take(sizeof(int) * 2);
        o.lr = take(sizeof(LigandRef) * cls[k].ligs.size());
        o.id = take(sizeof(uint32_t) * cls[k].ligs.size());
        o.res = take(sizeof(ResultDev) * nruns);
        o.bt = take(sizeof(float) * nruns * ntrace);
    }
    const size_t o_td = take(sizeof(int) * ADG_TRACE_WIDTH * tr_slots);
    const size_t o_tg = take(sizeof(float) * kGeneStride * tr_slots);
    const size_t o_te = take(sizeof(float) * tr_slots);
    if (off > ctx->arena_bytes) {
        CK(ctx, cudaStreamSynchronize(st));
        for (cudaStream_t s2 : ctx->class_streams) CK(ctx, cudaStreamSynchronize(s2));
        if (ctx->arena) cudaFree(ctx->arena);
        ctx->arena = nullptr;
        ctx->arena_bytes = 0;
        cudaError_t e = cudaMalloc(&ctx->arena, off);
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? ADG_ENOMEM : cuda_fail(ctx, e, "arena");
        ctx->arena_bytes = off;
    }
    char* A = (char*)ctx->arena;
    const MapsDev& M = rec->maps;
    const bool need_loop = p->max_gen > 0 && p->pop_size < p->nev;
    // streams: the first class runs on the context's stream, others on their own, joined by events
    while (ctx->class_streams.size() < cls.size()) {
        cudaStream_t s2;
        CK(ctx, cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
        ctx->class_streams.push_back(s2);
    }
    std::vector<std::vector<LigandRef>> lr(cls.size());
    std::vector<std::vector<uint32_t>> ids(cls.size());
    cudaEvent_t fork;
    CK(ctx, take_event(ctx, &fork));
    CK(ctx, cudaEventRecord(fork, st));
    for (size_t k = 0; k < cls.size(); ++k) {
        ClassRun& c = cls[k];
        const Offs& o = offs[k];
        c.stream = k == 0 ? st : ctx->class_streams[k];
        if (k > 0) CK(ctx, cudaStreamWaitEvent(c.stream, fork, 0));
        DockDev& D = c.D;
        D.ligs = (const LigandRef*)(A + o.lr);
        D.lig_id = (const uint32_t*)(A + o.id);
        D.nlig = (int)c.ligs.size();
        D.run0 = c.run0;
        D.pop_genes[0] = (float*)(A + o.g0);
        D.pop_genes[1] = (float*)(A + o.g1);
        D.pop_e[0] = (float*)(A + o.e0);
        D.pop_e[1] = (float*)(A + o.e1);
        D.evals = (unsigned long long*)(A + o.ev);
        D.gen_done = (int*)(A + o.gd);
        D.best_hist = (float*)(A + o.hist);
        D.stopped = (int*)(A + o.stop);
        D.best_trace = ntrace > 0 ? (float*)(A + o.bt) : nullptr;
        D.best_trace_len = ntrace;
        D.trace_ngen = tr_ngen;
        D.tr_dec = (int*)(A + o_td);
        D.tr_genes = (float*)(A + o_tg);
        D.tr_e = (float*)(A + o_te);
        c.d_active = (int*)(A + o.act);
        c.d_gen = (int*)(A + o.gen);
        c.d_res = (ResultDev*)(A + o.res);
        for (int i : c.ligs) {
            lr[k].push_back(ligs[i]->ref);
            ids[k].push_back(ligs[i]->stream_id >= 0 ? (uint32_t)ligs[i]->stream_id : p->lig_id + (uint32_t)i);
        }
        CK(ctx, cudaMemcpyAsync(A + o.lr, lr[k].data(), sizeof(LigandRef) * c.ligs.size(), cudaMemcpyHostToDevice,
                                c.stream));
        CK(ctx, cudaMemcpyAsync(A + o.id, ids[k].data(), sizeof(uint32_t) * c.ligs.size(), cudaMemcpyHostToDevice,
                                c.stream));
        ctx->stats.h2d_bytes += (int64_t)((sizeof(LigandRef) + sizeof(uint32_t)) * c.ligs.size());
        if (ctx->timing) {
            CK(ctx, take_event(ctx, &c.t0));
            CK(ctx, take_event(ctx, &c.t1));
        }
        const int nruns = (int)c.ligs.size() * c.S.nrun;
        if (ctx->use_graphs) {
            CK(ctx, build_class_graph(ctx, c, M, c.S, need_loop, ctx->timing, nruns));
            CK(ctx, cudaGraphLaunch(c.exec, c.stream));
        } else {
            cudaStream_t cs = c.stream;
            CK(ctx, cudaMemsetAsync(c.D.evals, 0, sizeof(unsigned long long) * 2 * nruns, cs));
            CK(ctx, cudaMemsetAsync(c.D.gen_done, 0, sizeof(int) * nruns, cs));
            CK(ctx, cudaMemsetAsync(c.D.stopped, 0, sizeof(int) * nruns, cs));
            if (c.D.best_trace)
                CK(ctx, cudaMemsetAsync(c.D.best_trace, 0xff, sizeof(float) * nruns * c.D.best_trace_len, cs));
            CK(ctx, launch_dock_init(cs, M, c.S, c.D, c.geo));
            if (ctx->timing) CK(ctx, cudaEventRecord(c.t0, cs));
        }
        ctx->stats.kernel_launches += 2;  // initial population and final poses; the loop adds 3 per generation
    }
    // host-driven generation loop (graphs off): every group advances four
    // generations between reads of its active-run count
    std::vector<int> host_gens(cls.size(), 0);
    if (!ctx->use_graphs) {
        std::vector<char> live(cls.size(), need_loop ? 1 : 0);
        std::vector<int> act(cls.size(), 0);
        for (;;) {
            bool any = false;
            for (size_t k = 0; k < cls.size(); ++k) {
                if (!live[k]) continue;
                any = true;
                ClassRun& c = cls[k];
                for (int q = 0; q < 4 && host_gens[k] < p->max_gen; ++q) {
                    const int gen = ++host_gens[k];
                    CK(ctx, cudaMemsetAsync(c.d_active, 0, sizeof(int), c.stream));
                    CK(ctx, launch_dock_generation(c.stream, M, c.S, c.D, c.geo, gen));
                    CK(ctx, launch_dock_count_active(c.stream, c.S, c.D, gen, c.d_active));
                }
                CK(ctx, cudaMemcpyAsync(&act[k], c.d_active, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
            }
            if (!any) break;
            for (size_t k = 0; k < cls.size(); ++k) {
                if (!live[k]) continue;
                CK(ctx, cudaStreamSynchronize(cls[k].stream));
                if (act[k] == 0 || host_gens[k] >= p->max_gen) live[k] = 0;
            }
        }
        for (size_t k = 0; k < cls.size(); ++k) {
            ClassRun& c = cls[k];
            if (ctx->timing) CK(ctx, cudaEventRecord(c.t1, c.stream));
            CK(ctx, launch_dock_finalize(c.stream, M, c.S, c.D, c.geo, c.d_res));
        }
    }
    std::vector<std::vector<ResultDev>> res(cls.size());
    std::vector<std::vector<float>> btr(cls.size());
    std::vector<int> gens_dev(cls.size(), 0);
    for (size_t k = 0; k < cls.size(); ++k) {
        ClassRun& c = cls[k];
        const long nruns = (long)c.ligs.size() * c.S.nrun;
        res[k].resize(nruns);
        CK(ctx, cudaMemcpyAsync(res[k].data(), c.d_res, sizeof(ResultDev) * nruns, cudaMemcpyDeviceToHost, c.stream));
        if (ctx->use_graphs) {
            CK(ctx, cudaMemcpyAsync(&gens_dev[k], c.d_gen, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
            ctx->stats.d2h_bytes += (int64_t)sizeof(int);
        } else {
            gens_dev[k] = host_gens[k];
        }
        ctx->stats.d2h_bytes += (int64_t)(sizeof(ResultDev) * nruns);
        if (ntrace > 0) {
            btr[k].resize((size_t)nruns * ntrace);
            CK(ctx, cudaMemcpyAsync(btr[k].data(), c.D.best_trace, sizeof(float) * nruns * ntrace,
                                    cudaMemcpyDeviceToHost, c.stream));
            ctx->stats.d2h_bytes += (int64_t)(sizeof(float) * nruns * ntrace);
        }
    }
    std::vector<int> tdec;
    std::vector<float> tg, te, init_g, init_e;
    for (size_t k = 0; k < cls.size(); ++k) CK(ctx, cudaStreamSynchronize(cls[k].stream));
    if (ctx->timing && need_loop) {
        // the groups' generation loops run concurrently: time their span, from
        // the first loop's start to the last one's end (both measured from the
        // fork every group waited on), over the longest group's generations
        float lo = 0.f, hi = 0.f;
        int rounds = 0;
        for (size_t k = 0; k < cls.size(); ++k) {
            float a = 0.f, b = 0.f;
            CK(ctx, cudaEventElapsedTime(&a, fork, cls[k].t0));
            CK(ctx, cudaEventElapsedTime(&b, fork, cls[k].t1));
            lo = k == 0 ? a : std::min(lo, a);
            hi = std::max(hi, b);
            rounds = std::max(rounds, gens_dev[k]);
        }
        ctx->stats.gen_kernel_ms += hi - lo;
        ctx->stats.gen_timed += rounds;
    }
    for (size_t k = 0; k < cls.size(); ++k) {
        ClassRun& c = cls[k];
        // generations executed by the device loop (the counter counts passes)
        const int ran = need_loop ? gens_dev[k] : 0;
        ctx->stats.gen_launches += ran;
        ctx->stats.kernel_launches += 3 * (int64_t)ran;
        if (c.t0) ctx->ev_free.push_back(c.t0);
        if (c.t1) ctx->ev_free.push_back(c.t1);
        if (c.exec) cudaGraphExecDestroy(c.exec);
    }
    ctx->ev_free.push_back(fork);
    if (trace) {
        // the single ligand's class ran on the context's stream
        const ClassRun& c = cls[0];
        const long nind = (long)p->nrun * p->pop_size;
        if (tr_slots > 0) {
            tdec.resize((size_t)tr_slots * ADG_TRACE_WIDTH);
            tg.resize((size_t)tr_slots * kGeneStride);
            te.resize(tr_slots);
            CK(ctx, cudaMemcpyAsync(tdec.data(), c.D.tr_dec, sizeof(int) * ADG_TRACE_WIDTH * tr_slots,
                                    cudaMemcpyDeviceToHost, st));
            CK(ctx, cudaMemcpyAsync(tg.data(), c.D.tr_genes, sizeof(float) * kGeneStride * tr_slots,
                                    cudaMemcpyDeviceToHost, st));
            CK(ctx, cudaMemcpyAsync(te.data(), c.D.tr_e, sizeof(float) * tr_slots, cudaMemcpyDeviceToHost, st));
        }
        if (trace->init_genes || trace->init_energies) {
            // generation 0 is deterministic: replay it into buffer 1 (free once
            // the results above are read; its evaluation counts are not needed)
            DockDev D1 = c.D;
            D1.pop_genes[0] = c.D.pop_genes[1];
            D1.pop_e[0] = c.D.pop_e[1];
            CK(ctx, launch_dock_init(st, M, c.S, D1, c.geo));
            init_g.resize((size_t)nind * kGeneStride);
            init_e.resize(nind);
            CK(ctx, cudaMemcpyAsync(init_g.data(), D1.pop_genes[0], sizeof(float) * nind * kGeneStride,
                                    cudaMemcpyDeviceToHost, st));
            CK(ctx, cudaMemcpyAsync(init_e.data(), D1.pop_e[0], sizeof(float) * nind, cudaMemcpyDeviceToHost, st));
        }
        CK(ctx, cudaStreamSynchronize(st));
    }
    for (size_t k = 0; k < cls.size(); ++k) {
        const ClassRun& c = cls[k];
        for (size_t li = 0; li < c.ligs.size(); ++li) {
            const int lig = c.ligs[li];
            const int G = 7 + ligs[lig]->ntors, N = ligs[lig]->natoms;
            for (int r = 0; r < c.S.nrun; ++r) {
                const int run = c.run0 + r;
                adg_result& o = out[(long)lig * p->nrun + run];
                const ResultDev& sr = res[k][(long)li * c.S.nrun + r];
                memset(&o, 0, sizeof(o));
                o.best_energy = sr.best_energy;
                o.generations = sr.generations;
                o.evals = sr.evals;
                for (int q = 0; q < G; ++q) o.genes[q] = sr.genes[q];
                for (int q = 0; q < 3 * N; ++q) o.xyz[q] = sr.xyz[q];
                if (ntrace > 0) {
                    // generations after the run's last repeat its final best energy
                    const float* src = btr[k].data() + ((long)li * c.S.nrun + r) * ntrace;
                    float* dst = best_trace + ((long)lig * p->nrun + run) * ntrace;
                    for (int q = 0; q < ntrace; ++q)
                        dst[q] = q < sr.generations ? src[q] : (q > 0 ? dst[q - 1] : sr.best_energy);
                }
            }
        }
    }
    if (trace) {
        const int G = 7 + ligs[0]->ntors;
        const long nind = (long)p->nrun * p->pop_size;
        if (trace->decisions && tr_slots)
            memcpy(trace->decisions, tdec.data(), sizeof(int) * ADG_TRACE_WIDTH * tr_slots);
        if (trace->energies && tr_slots) memcpy(trace->energies, te.data(), sizeof(float) * tr_slots);
        if (trace->genes)
            for (long q = 0; q < tr_slots; ++q)
                for (int k2 = 0; k2 < G; ++k2) trace->genes[q * G + k2] = tg[q * kGeneStride + k2];
        if (trace->init_genes)
            for (long q = 0; q < nind; ++q)
                for (int k2 = 0; k2 < G; ++k2) trace->init_genes[q * G + k2] = init_g[q * kGeneStride + k2];
        if (trace->init_energies) memcpy(trace->init_energies, init_e.data(), sizeof(float) * nind);
    }
    return ADG_OK;
}

}  // namespace

int adg_dock(adg_ctx* ctx, const adg_receptor* rec, const adg_ligand* const* ligs, int nlig,
             const adg_search_params* p, adg_result* out, adg_dock_trace* trace)
{
    return dock_impl(ctx, rec, ligs, nlig, p, out, trace, nullptr, 0);
}

int adg_dock_traced(adg_ctx* ctx, const adg_receptor* rec, const adg_ligand* const* ligs, int nlig,
                    const adg_search_params* p, adg_result* out, float* best_trace, int ntrace)
{
    if (ntrace <= 0 || !best_trace) return ADG_EINVAL;
    return dock_impl(ctx, rec, ligs, nlig, p, out, nullptr, best_trace, ntrace);
}

}  // extern "C"
