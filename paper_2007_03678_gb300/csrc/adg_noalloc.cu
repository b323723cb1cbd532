// adg_noalloc.cu -- adg_dock_noalloc: docking of one ligand for callers that
// cannot allocate memory.
//
// Some callers cannot call cudaMalloc: a host application whose own allocator
// owns all of the device memory and forbids libraries to allocate behind its
// back, or a latency-critical loop in which cudaMalloc / cudaFree (which may
// synchronize the device) would stall other work.  This entry point serves
// them: its working memory is the file-scope device array below, sized once
// for every GPU that loads the library, and the call itself allocates
// nothing (no cudaMalloc, cudaFree, host heap or allocating library call).
#include <mutex>
#include <stdint.h>
#include <string.h>

#include "adg_internal.h"

using namespace adg;

namespace {

// Working memory of adg_dock_noalloc: populations, evaluation counters and
// the result records.  Every GPU that loads the library holds it until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[ADG_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch per device (host code must not use the
// symbol itself: on the host it only stands in for the device array).
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

uint32_t prob_threshold(float p)
{
    if (p <= 0.f) return 0u;
    if (p >= 1.f) return 16777216u;
    return (uint32_t)((double)p * 16777216.0);
}

// Resolve the device address of the scratch array for `device` (current).
cudaError_t scratch_address(int device, void** out)
{
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[device] = p;
    }
    *out = g_scratch_addr[device];
    return cudaSuccess;
}

// Puts the caller's current device back when the call returns.
struct DeviceRestore {
    int prev = -1;
    ~DeviceRestore()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" int adg_dock_noalloc(const adg_receptor* rec, const adg_ligand* lig, const adg_search_params* p,
                                adg_result* out, void* stream)
{
    if (!rec || !lig || !p || !out) return ADG_EINVAL;
    if (p->nrun <= 0 || p->pop_size < 2 || p->pop_size > 65535 || p->nev < 0 || p->max_gen < 0 ||
        p->ls_max_iters < 0 || p->elitism < 0 || p->elitism > 1 || p->ls_method < 0 || p->ls_method > 2)
        return ADG_EINVAL;
    if (lig->device != rec->device || rec->device < 0 || rec->device >= kMaxDevices) return ADG_EINVAL;
    if (p->nrun > ADG_NOALLOC_MAX_RUNS || (long)p->nrun * p->pop_size > ADG_NOALLOC_MAX_INDIVIDUALS)
        return ADG_ETOOBIG;
    cudaStream_t st = (cudaStream_t)stream;
    DeviceRestore restore;
    if (cudaGetDevice(&restore.prev) != cudaSuccess) return ADG_ECUDA;
    if (cudaSetDevice(rec->device) != cudaSuccess) return ADG_ECUDA;
    void* base = nullptr;
    if (scratch_address(rec->device, &base) != cudaSuccess) return ADG_ECUDA;
    // carve the scratch array
    const long nruns = p->nrun, nind = nruns * p->pop_size;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    const size_t o_g0 = take(sizeof(float) * nind * kGeneStride), o_g1 = take(sizeof(float) * nind * kGeneStride);
    const size_t o_e0 = take(sizeof(float) * nind), o_e1 = take(sizeof(float) * nind);
    const size_t o_ev = take(sizeof(unsigned long long) * 2 * nruns);
    const size_t o_gd = take(sizeof(int) * nruns);
    const size_t o_hist = take(sizeof(float) * 10 * nruns);
    const size_t o_stop = take(sizeof(int) * nruns);
    const size_t o_act = take(sizeof(int) * 2);
    const size_t o_lr = take(sizeof(LigandRef));
    const size_t o_id = take(sizeof(uint32_t));
    const size_t o_res = take(sizeof(adg_result) * nruns);
    if (off > ADG_NOALLOC_SCRATCH_BYTES) return ADG_ETOOBIG;
    char* A = (char*)base;
    SearchDev S;
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
    DockDev D;
    D.ligs = (const LigandRef*)(A + o_lr);
    D.lig_id = (const uint32_t*)(A + o_id);
    D.nlig = 1;
    D.run0 = 0;
    D.pop_genes[0] = (float*)(A + o_g0);
    D.pop_genes[1] = (float*)(A + o_g1);
    D.pop_e[0] = (float*)(A + o_e0);
    D.pop_e[1] = (float*)(A + o_e1);
    D.evals = (unsigned long long*)(A + o_ev);
    D.gen_done = (int*)(A + o_gd);
    D.best_hist = (float*)(A + o_hist);
    D.stopped = (int*)(A + o_stop);
    D.best_trace = nullptr;
    D.best_trace_len = 0;
    D.trace_ngen = 0;
    D.tr_dec = nullptr;
    D.tr_genes = nullptr;
    D.tr_e = nullptr;
    int* d_active = (int*)(A + o_act);
    adg_result* d_res = (adg_result*)(A + o_res);
    const Geo geo = make_geo(lig->apl, lig->nslots, lig->bytes);
    const MapsDev& M = rec->maps;
    // host values live on this stack frame until the final synchronize below
    const LigandRef lr = lig->ref;
    const uint32_t id = lig->stream_id >= 0 ? (uint32_t)lig->stream_id : p->lig_id;
    int active = 0;
#define NA_CK(call)                                 \
    do {                                            \
        if ((call) != cudaSuccess) return ADG_ECUDA; \
    } while (0)
    NA_CK(cudaMemcpyAsync(A + o_lr, &lr, sizeof(lr), cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(A + o_id, &id, sizeof(id), cudaMemcpyHostToDevice, st));
    // the array keeps the previous call's contents: clear what must start at zero
    NA_CK(cudaMemsetAsync(D.evals, 0, sizeof(unsigned long long) * 2 * nruns, st));
    NA_CK(cudaMemsetAsync(D.gen_done, 0, sizeof(int) * nruns, st));
    NA_CK(cudaMemsetAsync(D.stopped, 0, sizeof(int) * nruns, st));
    NA_CK(launch_dock_init(st, M, S, D, geo));
    const bool need_more = p->max_gen > 0 && p->pop_size < p->nev;
    int gen = 0;
    while (need_more) {
        int last = gen;
        for (int c = 0; c < 4 && gen < p->max_gen; ++c) {
            ++gen;
            NA_CK(cudaMemsetAsync(d_active, 0, sizeof(int), st));
            NA_CK(launch_dock_generation(st, M, S, D, geo, gen));
            NA_CK(launch_dock_count_active(st, S, D, gen, d_active));
            last = gen;
        }
        NA_CK(cudaMemcpyAsync(&active, d_active, sizeof(int), cudaMemcpyDeviceToHost, st));
        NA_CK(cudaStreamSynchronize(st));
        if (active == 0 || last >= p->max_gen) break;
    }
    NA_CK(launch_dock_finalize_abi(st, M, S, D, geo, d_res));
    NA_CK(cudaMemcpyAsync(out, d_res, sizeof(adg_result) * nruns, cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
#undef NA_CK
    return ADG_OK;
}
