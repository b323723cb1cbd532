// adg_kernels.cu -- sm_103a kernels of the docking hot path (arXiv 2007.03678).
//
// One warp owns one individual (one genotype): lanes own atoms for the pose
// and the grid gather, lanes own intramolecular pairs for the pair terms,
// and warp shuffles reduce the energy and the genotype gradient.  A whole
// GA generation of an individual -- selection, crossover, mutation, the
// offspring evaluation and its local search (Solis-Wets or ADADELTA) -- runs
// inside that one warp, so a generation of every run of a ligand group is
// one launch.  The receptor maps are packed per atom type as one 32-byte
// record per node, (M_t, M_elec, M_desolv, 0) at x and at x + 1, so that a
// trilinear gather is four 32-byte loads served from L2 (a 64^3 receptor is
// 59 MB packed, inside the 126 MB L2).
#include <math.h>
#include <stdint.h>

#include "adg_internal.h"

namespace adg {

#define FULL_MASK 0xffffffffu

// Minimum resident blocks per SM the warp-per-individual kernels are
// compiled for (bounds their registers: 2 blocks of 12 warps -> 85 per thread).
#ifndef ADG_MIN_BLOCKS
#define ADG_MIN_BLOCKS 2
#endif

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of two 32x32 multiplies
// whose high halves are xored into the other words with the round key; the
// key is bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// Stream layout: counter = (ligand id, run << 16 | individual, generation,
// purpose << 20 | block), key = 64-bit seed.
enum { P_INIT = 1, P_SELECT = 2, P_MUTATE = 3, P_LSPICK = 4, P_LS = 5 };

struct Rng {
    uint32_t k0, k1, lig, run, ind, gen;
    __device__ __forceinline__ uint4 block(int purpose, int blk) const
    {
        return philox(make_uint4(lig, (run << 16) | ind, gen, ((uint32_t)purpose << 20) | (uint32_t)blk), k0, k1);
    }
};

__device__ __forceinline__ float u01(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }
__device__ __forceinline__ float u01_open0(uint32_t x) { return (float)((x >> 8) + 1u) * (1.0f / 16777216.0f); }
__device__ __forceinline__ int uindex(uint32_t x, int n) { return (int)(((unsigned long long)x * (unsigned)n) >> 32); }
__device__ __forceinline__ bool ptest(uint32_t x, uint32_t thr) { return (x >> 8) < thr; }
__device__ __forceinline__ uint32_t word(uint4 w, int i) { return i == 0 ? w.x : i == 1 ? w.y : i == 2 ? w.z : w.w; }

__global__ void k_philox(const uint32_t* __restrict__ ctr, int n, uint32_t k0, uint32_t k1, uint32_t* __restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint4 c = reinterpret_cast<const uint4*>(ctr)[i];
    reinterpret_cast<uint4*>(out)[i] = philox(c, k0, k1);
}

cudaError_t launch_philox(cudaStream_t st, const uint32_t* ctr, int n, uint32_t k0, uint32_t k1, uint32_t* out)
{
    if (n > 0) k_philox<<<(n + 255) / 256, 256, 0, st>>>(ctr, n, k0, k1, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ maps (a0)
struct MapConst {
    double c12[ADG_NTYPES][ADG_NTYPES], c6[ADG_NTYPES][ADG_NTYPES], c10[ADG_NTYPES][ADG_NTYPES];
    double solpar[ADG_NTYPES], vol[ADG_NTYPES];
    double w_desolv, qasp, inv_2s2, w_elec_coul;
    double ms_A, ms_B, ms_k, ms_lb;
    float r_min, rmin2, e_cap, r_on, r_off;
    float ox, oy, oz, h;
    int nx, ny, nz;
};

// One thread per grid node; receptor atoms stream through shared memory.
// The terms are evaluated in FP64 (the maps are built once per receptor, and
// near receptor atoms the 12-6 / 12-10 terms reach 1e5 kcal/mol, where FP32
// powers of 1/r lose the digits the interpolation later needs); stored FP32.
__global__ void __launch_bounds__(256) k_maps_build(MapConst C, int nrec, const float4* __restrict__ rxyzq,
                                                    const int* __restrict__ rtype, float* __restrict__ maps)
{
    __shared__ float4 sa[256];
    __shared__ int st[256];
    const long npt = (long)C.nx * C.ny * C.nz;
    const long node = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int ix = (int)(node % C.nx), iy = (int)((node / C.nx) % C.ny), iz = (int)(node / ((long)C.nx * C.ny));
    const double px = (double)C.ox + ix * (double)C.h, py = (double)C.oy + iy * (double)C.h,
                 pz = (double)C.oz + iz * (double)C.h;
    double acc[ADG_NMAPS];
#pragma unroll
    for (int m = 0; m < ADG_NMAPS; ++m) acc[m] = 0.0;
    const double roff2 = (double)C.r_off * C.r_off, rmin = C.r_min, inv_2s2 = C.inv_2s2;
    for (int base = 0; base < nrec; base += 256) {
        __syncthreads();
        if (base + threadIdx.x < nrec) {
            sa[threadIdx.x] = rxyzq[base + threadIdx.x];
            st[threadIdx.x] = rtype[base + threadIdx.x];
        }
        __syncthreads();
        const int cnt = min(256, nrec - base);
        if (node >= npt) continue;
        for (int j = 0; j < cnt; ++j) {
            const float4 a = sa[j];
            const double dx = px - a.x, dy = py - a.y, dz = pz - a.z;
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 >= roff2) continue;
            const double r = sqrt(r2);
            double sw = 1.0;
            if (r > C.r_on) {
                const double u = (r - C.r_on) / ((double)C.r_off - C.r_on);
                sw = 1.0 - 3.0 * u * u + 2.0 * u * u * u;
            }
            const double rr = r < rmin ? rmin : r;
            const double rr2 = rr * rr;
            const double G = exp(-rr2 * inv_2s2);
            const double ri2 = 1.0 / rr2;
            const double ri6 = ri2 * ri2 * ri2, ri12 = ri6 * ri6, ri10 = ri6 * ri2 * ri2;
            const int tj = st[j];
            const double qj = a.w, aqj = fabs((double)a.w);
#pragma unroll
            for (int t = 0; t < ADG_NTYPES; ++t) {
                double e = C.c12[t][tj] * ri12 - C.c6[t][tj] * ri6 - C.c10[t][tj] * ri10;
                e = fmin(e, (double)C.e_cap);
                e += C.w_desolv * (C.solpar[t] * C.vol[tj] + (C.solpar[tj] + C.qasp * aqj) * C.vol[t]) * G;
                acc[t] += sw * e;
            }
            const double eps = C.ms_A + C.ms_B / (1.0 + C.ms_k * exp(-C.ms_lb * rr));
            acc[ADG_MAP_ELEC] += sw * C.w_elec_coul * qj / (eps * rr);
            acc[ADG_MAP_DESOLV] += sw * C.w_desolv * C.qasp * C.vol[tj] * G;
        }
    }
    if (node >= npt) return;
#pragma unroll
    for (int t = 0; t < ADG_NTYPES; ++t) acc[t] = fmin(acc[t], (double)C.e_cap);
#pragma unroll
    for (int m = 0; m < ADG_NMAPS; ++m) maps[m * npt + node] = (float)acc[m];
}

static void lj_coefs(const adg_forcefield& ff, int ti, int tj, double* c12, double* c6, double* c10)
{
    // generalised n-m well with minimum -eps at r0: C_n = m/(n-m) eps r0^n, C_m = n/(n-m) eps r0^m
    const bool hb = (ff.hb_donor[ti] && ff.hb_acceptor[tj]) || (ff.hb_donor[tj] && ff.hb_acceptor[ti]);
    double r0, eps, w;
    int m;
    if (hb) {
        const int acc = ff.hb_acceptor[tj] ? tj : ti;
        r0 = ff.hb_R[acc];
        eps = ff.hb_eps[acc];
        w = ff.w_hb;
        m = 10;
    } else {
        r0 = 0.5 * ((double)ff.Rii[ti] + ff.Rii[tj]);
        eps = sqrt((double)ff.epsii[ti] * ff.epsii[tj]);
        w = ff.w_vdw;
        m = 6;
    }
    double rn = 1.0, rm = 1.0;
    for (int k = 0; k < 12; ++k) rn *= r0;
    for (int k = 0; k < m; ++k) rm *= r0;
    *c12 = w * (double)m / (12 - m) * eps * rn;
    const double cm = w * 12.0 / (12 - m) * eps * rm;
    *c6 = m == 6 ? cm : 0.0;
    *c10 = m == 10 ? cm : 0.0;
}

void pair_coefs(const adg_forcefield& ff, int ti, int tj, float* c12, float* c6, float* c10)
{
    double a, b, c;
    lj_coefs(ff, ti, tj, &a, &b, &c);
    *c12 = (float)a;
    *c6 = (float)b;
    *c10 = (float)c;
}

cudaError_t launch_maps_build(cudaStream_t st, const adg_forcefield& ff, const adg_grid_desc& g, int nrec,
                              const float4* rec_xyzq, const int* rec_type, float* maps_out)
{
    MapConst C;
    for (int t = 0; t < ADG_NTYPES; ++t)
        for (int u = 0; u < ADG_NTYPES; ++u) lj_coefs(ff, t, u, &C.c12[t][u], &C.c6[t][u], &C.c10[t][u]);
    for (int t = 0; t < ADG_NTYPES; ++t) {
        C.solpar[t] = ff.solpar[t];
        C.vol[t] = ff.vol[t];
    }
    C.w_desolv = ff.w_desolv;
    C.qasp = ff.qasp;
    C.inv_2s2 = 1.0 / (2.0 * (double)ff.sigma * ff.sigma);
    C.w_elec_coul = (double)ff.w_elec * ff.coulomb;
    C.ms_A = ff.ms_A;
    C.ms_B = (double)ff.ms_eps0 - ff.ms_A;
    C.ms_k = ff.ms_k;
    C.ms_lb = (double)ff.ms_lambda * ((double)ff.ms_eps0 - ff.ms_A);
    C.r_min = ff.r_min;
    C.rmin2 = ff.r_min * ff.r_min;
    C.e_cap = ff.e_cap;
    C.r_on = ff.map_r_on;
    C.r_off = ff.map_r_off;
    C.ox = g.origin[0];
    C.oy = g.origin[1];
    C.oz = g.origin[2];
    C.h = g.spacing;
    C.nx = g.n[0];
    C.ny = g.n[1];
    C.nz = g.n[2];
    const long npt = (long)g.n[0] * g.n[1] * g.n[2];
    k_maps_build<<<(unsigned)((npt + 255) / 256), 256, 0, st>>>(C, nrec, rec_xyzq, rec_type, maps_out);
    return cudaGetLastError();
}

// The caller's [map][z][y][x] maps -> per atom type t and node i the record
// packed[2 (t npt + i)], packed[2 (t npt + i) + 1] = the node and its x + 1 neighbour.
__global__ void k_pack_maps(const float* __restrict__ maps, long npt, int nx, float4* __restrict__ packed)
{
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npt) return;
    const long i1 = (i % nx == nx - 1) ? i : i + 1;  // the x + 1 neighbour (the last node repeats itself)
    const float e = maps[ADG_MAP_ELEC * npt + i], d = maps[ADG_MAP_DESOLV * npt + i];
    const float e1 = maps[ADG_MAP_ELEC * npt + i1], d1 = maps[ADG_MAP_DESOLV * npt + i1];
#pragma unroll
    for (int t = 0; t < ADG_NTYPES; ++t) {
        packed[2 * (t * npt + i)] = make_float4(maps[t * npt + i], e, d, 0.f);
        packed[2 * (t * npt + i) + 1] = make_float4(maps[t * npt + i1], e1, d1, 0.f);
    }
}

cudaError_t launch_pack_maps(cudaStream_t st, const float* maps, const adg_grid_desc& g, float4* packed)
{
    const long npt = (long)g.n[0] * g.n[1] * g.n[2];
    k_pack_maps<<<(unsigned)((npt + 255) / 256), 256, 0, st>>>(maps, npt, g.n[0], packed);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ warp scoring
// Per-warp views into the dynamic shared memory of the block.
struct WarpView {
    float4* xyz;   // posed coordinates [na] (internal atom order), then the pad atom
    float4* f;     // row forces per atom, then prefix sums of the total force [na]; f[na]: sink
    float4* pm;    // the force gather's (sum c_p, sum c_p x_partner) per atom, then prefix sums of the moments (x - t) x f [na]
    float4* W;     // fragment transforms, rows 3f..3f+2 = (R row, t) [52]
    float* genes;  // current genotype [32]
    float* cand;   // trial genotype [32]
    float* best;   // best genotype of a local search [32]
    float* c;      // (dE/dr)/r per pair slot [nslots]
};

__device__ __forceinline__ WarpView warp_view(int na, int nslots, int lig_bytes)
{
    extern __shared__ float4 dyn_smem4[];
    float* base = reinterpret_cast<float*>(reinterpret_cast<char*>(dyn_smem4) + lig_bytes) +
                  (size_t)(threadIdx.x >> 5) * warp_smem_floats(na, nslots);
    WarpView v;
    v.xyz = reinterpret_cast<float4*>(base);
    v.f = reinterpret_cast<float4*>(base + 4 * na + 4);
    v.pm = reinterpret_cast<float4*>(base + 8 * na + 8);
    v.W = reinterpret_cast<float4*>(base + 12 * na + 8);
    v.genes = base + 12 * na + 216;
    v.cand = v.genes + 32;
    v.best = v.cand + 32;
    v.c = v.best + 32;
    // the pad atom: the row atom of empty pair slots (origin, zero charge);
    // read only after the __syncwarp that ends every pose
    if ((threadIdx.x & 31) == 0) v.xyz[na] = make_float4(0.f, 0.f, 0.f, 0.f);
    return v;
}

// Copy the block's ligand blob (header, pair slots, gather program) into the
// front of the dynamic shared memory; every thread of the block calls this
// before any warp leaves.  lig_bytes == 0 keeps the ligand in global memory.
// With the form fixed at compile time (FORM = 1 staged, 0 global; -1 chosen
// by lig_bytes) the returned pointers have one state space, so the compiler
// addresses the staged ligand with 32-bit shared-memory loads instead of
// generic ones.
template <int FORM = -1>
__device__ __forceinline__ LigandRef stage_ligand(const LigandRef& g, int lig_bytes)
{
    extern __shared__ float4 dyn_smem4[];
    if (FORM == 0 || (FORM < 0 && lig_bytes == 0)) return g;
    const int n16 = g.hdr->blob_bytes / 16;
    const int4* src = reinterpret_cast<const int4*>(g.hdr);
    int4* dst = reinterpret_cast<int4*>(dyn_smem4);
    for (int i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = __ldg(src + i);
    __syncthreads();
    const char* b = reinterpret_cast<const char*>(dyn_smem4);
    const LigandDev* L = reinterpret_cast<const LigandDev*>(b);
    LigandRef r;
    r.hdr = L;
    r.pairs.pk = reinterpret_cast<const float4*>(b + L->off_pk);
    r.pairs.gent = reinterpret_cast<const uint32_t*>(b + L->off_gent);
    return r;
}

// Two-wide FP32 arithmetic: one instruction computes both halves of a float2
// (each rounded to nearest, as the scalar operation would be).
__device__ __forceinline__ float2 v2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 s2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

// The special-function unit's approximations with subnormals flushed: one
// instruction each.  The pair terms never meet a subnormal (r >= sqrt(rmin2),
// r bounded by the ligand's extent), and without .ftz each call carries the
// scaling steps that preserve subnormal inputs and outputs.
__device__ __forceinline__ float ex2_ftz(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_ftz(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
constexpr float kLog2e = 1.4426950408889634f;

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
    return v;
}

// Genotype g (shared memory, 7+T floats) -> posed coordinates in ws.xyz.
// Applying the torsions deepest first about their reference axes and then
// x' = R(q/|q|)(x - c) + t is, per rigid fragment, one affine map
// W_f = W_parent(f) * Rot_k(f): the rigid-body map for the root fragment,
// composed down the fragment tree one level at a time (three lanes per
// fragment, one per row, or one lane per fragment past 10 fragments), then
// applied once to each atom.  ANY: APL may exceed the ligand's own atoms per
// lane (the layout width is then read from the ligand).
template <int APL, bool ANY = false>
__device__ __forceinline__ void warp_pose(const LigandDev* __restrict__ L, const float* g, const WarpView& ws, int lane,
                                          float4 (&xo)[APL], int (&to)[APL])
{
    const int N = L->natoms, NF = L->nfrag;
    // Up to 10 fragments: lane 3f + i builds row i of fragment f's map (the
    // rows are independent, each needs the whole local map); otherwise lane f
    // builds all three rows.  Either way each row is the same arithmetic.
    const bool by_row = NF <= 10;
    const int f = by_row ? lane / 3 : lane;
    const int ri = by_row ? lane - 3 * f : 0;
    float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0;  // fragment f's local map: rotation rows | translation
    if (f < NF) {
        // fragment 0: x' = R(q/|q|)(x - c) + t; fragment f > 0: the rotation by
        // theta about its torsion axis through o, x' = R(x - o) + o, with R from
        // the unit quaternion (cos theta/2, sin theta/2 u).  One
        // quaternion-to-matrix path for both, so the lanes do not diverge.
        const int k = f > 0 ? L->ftor[f] : 0;
        float s, c;
        sincosf(f > 0 ? 0.5f * g[7 + k] : 0.f, &s, &c);
        const float4 u = L->tax[k], o = L->tpt[k];
        float qw = c, qx = s * u.x, qy = s * u.y, qz = s * u.z;
        float px = o.x, py = o.y, pz = o.z, tx = o.x, ty = o.y, tz = o.z;
        if (f == 0) {
            qw = g[3]; qx = g[4]; qy = g[5]; qz = g[6];
            const float qi = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
            qw *= qi; qx *= qi; qy *= qi; qz *= qi;
            px = L->cx; py = L->cy; pz = L->cz;
            tx = g[0]; ty = g[1]; tz = g[2];
        }
        const float R00 = 1.f - 2.f * (qy * qy + qz * qz), R01 = 2.f * (qx * qy - qw * qz), R02 = 2.f * (qx * qz + qw * qy);
        const float R10 = 2.f * (qx * qy + qw * qz), R11 = 1.f - 2.f * (qx * qx + qz * qz), R12 = 2.f * (qy * qz - qw * qx);
        const float R20 = 2.f * (qx * qz - qw * qy), R21 = 2.f * (qy * qz + qw * qx), R22 = 1.f - 2.f * (qx * qx + qy * qy);
        r0 = make_float4(R00, R01, R02, tx - (R00 * px + R01 * py + R02 * pz));
        r1 = make_float4(R10, R11, R12, ty - (R10 * px + R11 * py + R12 * pz));
        r2 = make_float4(R20, R21, R22, tz - (R20 * px + R21 * py + R22 * pz));
        if (f == 0) {
            if (by_row) {
                ws.W[ri] = ri == 0 ? r0 : (ri == 1 ? r1 : r2);
            } else {
                ws.W[0] = r0;
                ws.W[1] = r1;
                ws.W[2] = r2;
            }
        }
    }
    __syncwarp();
    const int maxlev = L->maxlev;
    const int mylev = (f > 0 && f < NF) ? L->flev[f] : -1;
    for (int lev = 1; lev <= maxlev; ++lev) {
        if (mylev == lev) {
            const int p = L->fpar[f];
            // row of W_parent times the local map, two columns per two-wide operation
            const float2 r0a = v2(r0.x, r0.y), r0b = v2(r0.z, r0.w), r1a = v2(r1.x, r1.y), r1b = v2(r1.z, r1.w),
                         r2a = v2(r2.x, r2.y), r2b = v2(r2.z, r2.w);
            auto row = [&](const float4 P) {
                const float2 a = __ffma2_rn(s2(P.z), r2a, __ffma2_rn(s2(P.y), r1a, __fmul2_rn(s2(P.x), r0a)));
                const float2 b = __ffma2_rn(s2(P.z), r2b, __ffma2_rn(s2(P.y), r1b, __fmul2_rn(s2(P.x), r0b)));
                return make_float4(a.x, a.y, b.x, b.y + P.w);
            };
            if (by_row) {
                ws.W[3 * f + ri] = row(ws.W[3 * p + ri]);
            } else {
                const float4 p0 = ws.W[3 * p], p1 = ws.W[3 * p + 1], p2 = ws.W[3 * p + 2];
                ws.W[3 * f] = row(p0);
                ws.W[3 * f + 1] = row(p1);
                ws.W[3 * f + 2] = row(p2);
            }
        }
        __syncwarp();
    }
#pragma unroll
    for (int j = 0; j < APL; ++j) {
        const int a = lane + 32 * j;  // the atom index of depth-first position apl lane + j
        const int apl = ANY ? L->apl : APL;
        xo[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        to[j] = 0;
        if (j < apl && apl * lane + j < N) {
            const float4 r = L->ref[a];
            const int tf = L->tf[a], f = tf >> 8;
            const float4 w0 = ws.W[3 * f], w1 = ws.W[3 * f + 1], w2 = ws.W[3 * f + 2];
            xo[j] = make_float4(w0.x * r.x + w0.y * r.y + w0.z * r.z + w0.w, w1.x * r.x + w1.y * r.y + w1.z * r.z + w1.w,
                                w2.x * r.x + w2.y * r.y + w2.z * r.z + w2.w, r.w);  // .w: the charge
            to[j] = tf & 255;
            ws.xyz[a] = xo[j];
        }
    }
    __syncwarp();
}

template <int APL, bool ANY>
__device__ __forceinline__ void warp_pose(const LigandDev* __restrict__ L, const float* g, const WarpView& ws, int lane)
{
    float4 xo[APL];
    int to[APL];
    warp_pose<APL, ANY>(L, g, ws, lane, xo, to);
}

// Both x-corners of a cell edge, one 32-byte record: (M_t, M_e, M_d, 0) at x and at x + 1.
__device__ __forceinline__ void ldg_pair(const float4* p, float4& a, float4& b)
{
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
}

// Intermolecular energy of one atom: trilinear interpolation of
// M_t + q M_e + |q| M_d at the point clamped into the box, plus k_out d^2
// outside it; gradient accumulated into (gx, gy, gz).
template <bool GRAD>
__device__ __forceinline__ float atom_inter(const MapsDev& M, float k_out, int t, float q, float x, float y, float z,
                                            float& gx, float& gy, float& gz)
{
    // the point clamped into the box and its distance outside, per axis
    const float xc = fminf(fmaxf(x, M.ox), M.hx), yc = fminf(fmaxf(y, M.oy), M.hy), zc = fminf(fmaxf(z, M.oz), M.hz);
    const float ex = x - xc, ey = y - yc, ez = z - zc;
    const float pen = ex * ex + ey * ey + ez * ez;
    const float pgx = 2.f * k_out * ex, pgy = 2.f * k_out * ey, pgz = 2.f * k_out * ez;
    const bool clx = ex != 0.f, cly = ey != 0.f, clz = ez != 0.f;
    const float ux = (xc - M.ox) * M.inv_h, uy = (yc - M.oy) * M.inv_h, uz = (zc - M.oz) * M.inv_h;
    int ix = min(max((int)floorf(ux), 0), M.nx - 2);
    int iy = min(max((int)floorf(uy), 0), M.ny - 2);
    int iz = min(max((int)floorf(uz), 0), M.nz - 2);
    // The fractions are taken from the cell's own corner node, not from u:
    // u carries the rounding of (x - o) / h at the scale of the whole box (a
    // few 1e-6 of a cell), which near a capped map value (slopes up to
    // 1e5 kcal/mol per 0.375 A) is worth 1e-2 kcal/mol.  x - node is exact
    // (the node o + i h is representable and within a cell of x), and one
    // residual step rounds (x - node) / h to within an ulp of f.
    const float dx = xc - fmaf((float)ix, M.h, M.ox), dy = yc - fmaf((float)iy, M.h, M.oy),
                dz = zc - fmaf((float)iz, M.h, M.oz);
    float fx = dx * M.inv_h, fy = dy * M.inv_h, fz = dz * M.inv_h;
    fx = fmaf(fmaf(-fx, M.h, dx), M.inv_h, fx);
    fy = fmaf(fmaf(-fy, M.h, dy), M.inv_h, fy);
    fz = fmaf(fmaf(-fz, M.h, dz), M.inv_h, fz);
    const int nxy = M.nx * M.ny;
    const float4* p = M.packed + 2 * ((long)t * nxy * M.nz + (iz * nxy + iy * M.nx + ix));
    const float aq = fabsf(q);
    float4 c000, c100, c010, c110, c001, c101, c011, c111;
    ldg_pair(p, c000, c100);
    ldg_pair(p + 2 * M.nx, c010, c110);
    ldg_pair(p + 2 * nxy, c001, c101);
    ldg_pair(p + 2 * (nxy + M.nx), c011, c111);
    const float v000 = c000.x + q * c000.y + aq * c000.z, v100 = c100.x + q * c100.y + aq * c100.z;
    const float v010 = c010.x + q * c010.y + aq * c010.z, v110 = c110.x + q * c110.y + aq * c110.z;
    const float v001 = c001.x + q * c001.y + aq * c001.z, v101 = c101.x + q * c101.y + aq * c101.z;
    const float v011 = c011.x + q * c011.y + aq * c011.z, v111 = c111.x + q * c111.y + aq * c111.z;
    const float a00 = v000 + fx * (v100 - v000), a10 = v010 + fx * (v110 - v010);
    const float a01 = v001 + fx * (v101 - v001), a11 = v011 + fx * (v111 - v011);
    const float b0 = a00 + fy * (a10 - a00), b1 = a01 + fy * (a11 - a01);
    const float val = b0 + fz * (b1 - b0);
    if (GRAD) {
        const float dx0 = (v100 - v000) + fy * ((v110 - v010) - (v100 - v000));
        const float dx1 = (v101 - v001) + fy * ((v111 - v011) - (v101 - v001));
        const float dvx = dx0 + fz * (dx1 - dx0);
        const float dvy = (a10 - a00) + fz * ((a11 - a01) - (a10 - a00));
        const float dvz = b1 - b0;
        gx += (clx ? 0.f : dvx * M.inv_h) + pgx;
        gy += (cly ? 0.f : dvy * M.inv_h) + pgy;
        gz += (clz ? 0.f : dvz * M.inv_h) + pgz;
    }
    return val + k_out * pen;
}

struct ScoreOut {
    float e;           // total energy (all lanes)
    float gtan;        // lane d < 6+T: tangent gradient component d
    float tx, ty, tz;  // torque (all lanes)
};

// Energy (and gradient) of the genotype in shared memory `g`.
//  1. pose (lanes own atoms), 2. intermolecular gather (lanes own atoms),
//  3. pair terms (lanes own rows of pair slots; the gradient pass stores
//     c_p = (dE/dr)/r per slot and sums each row owner's force in
//     registers), 4. force gather of the partner sides from c_p (no
//     atomics: each atom belongs to one lane's gather list), 5. prefix sums
//     over the depth-first atom order and one transposed warp reduction of
//     dE/dt, the torque and every dE/dtheta.
template <int APL, bool GRAD>
__device__ __forceinline__ ScoreOut warp_score(const LigandDev* __restrict__ L, const PairsDev& P, const MapsDev& M,
                                               const float* g, const WarpView& ws, int lane)
{
    float4 xo[APL];  // this lane's posed atoms (charge in .w) and their types
    int to[APL];
    warp_pose<APL>(L, g, ws, lane, xo, to);
    const int N = L->natoms, T = L->ntors;
    const float k_out = L->k_out;
    float e = 0.f;
    float fxr[APL], fyr[APL], fzr[APL];
#pragma unroll
    for (int j = 0; j < APL; ++j) {
        fxr[j] = fyr[j] = fzr[j] = 0.f;
        const int a = lane + 32 * j;
        if (APL * lane + j < N) {  // the atom of depth-first position APL lane + j
            const float4 x = xo[j];
            e += atom_inter<GRAD>(M, k_out, to[j], x.w, x.x, x.y, x.z, fxr[j], fyr[j], fzr[j]);
            if (GRAD) {
                ws.f[a] = make_float4(0.f, 0.f, 0.f, 0.f);
                ws.pm[a] = make_float4(0.f, 0.f, 0.f, 0.f);  // atoms the gather does not reach
            }
        }
    }
    if (GRAD) __syncwarp();  // rows below store into f of atoms other lanes cleared
    // intramolecular pairs, two slots per step in two-wide FP32 arithmetic
    // (one instruction for both); the force on a row owner accumulates in
    // registers and is stored at the row's end
    const float cap = L->e_cap, rmin2 = L->rmin2, msA = L->ms_A, msB = L->ms_B, msk = L->ms_k, mslb = L->ms_lb;
    const float inv_2s2 = L->inv_2s2, inv_s2 = L->inv_s2, wq = L->wq;
    // exp(-lambda r) and exp(-r^2 / 2 sigma^2) as powers of two
    const float kex = -mslb * kLog2e, kgs = -inv_2s2 * kLog2e;
    const int nsteps = L->nsteps;  // even
    float rfx = 0.f, rfy = 0.f, rfz = 0.f;
    float4 xr = make_float4(0.f, 0.f, 0.f, 0.f);  // atom i of the current row
    float2 e2 = s2(0.f);
    for (int stp = 0; stp < nsteps; stp += 2) {
        const int ia = stp * 32 + lane, ib = ia + 32;
        // (c12, cm) of both slots, then (cd, ij) of both slots
        const float4 pa = P.pk[ia], pb = P.pk[ib];
        const int ija = __float_as_int(pb.z), ijb = __float_as_int(pb.w);
        if (ija & kPairRowStart) xr = ws.xyz[ija & 255];
        const float4 xia = xr, xja = ws.xyz[(ija >> 16) & 127];
        if (ijb & kPairRowStart) xr = ws.xyz[ijb & 255];
        const float4 xib = xr, xjb = ws.xyz[(ijb >> 16) & 127];
        // differences one slot at a time, so each lands in its half of a pair
        const float2 dx = v2(xia.x - xja.x, xib.x - xjb.x);
        const float2 dy = v2(xia.y - xja.y, xib.y - xjb.y);
        const float2 dz = v2(xia.z - xja.z, xib.z - xjb.z);
        const float2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
        const float2 c12 = v2(pa.x, pa.y), cm = v2(pa.z, pa.w), cd = v2(pb.x, pb.y);
        // cq = wq q_i q_j (0 on an empty slot: its row atom is the uncharged pad)
        const float2 cq = v2(wq * xia.w * xja.w, wq * xib.w * xjb.w);
        const bool fla = r2.x < rmin2, flb = r2.y < rmin2;
        const float2 rr2 = v2(fla ? rmin2 : r2.x, flb ? rmin2 : r2.y);
        const float2 ri = v2(rsqrt_ftz(rr2.x), rsqrt_ftz(rr2.y));
        const float2 r = mul2(rr2, ri);
        const float2 ri2 = mul2(ri, ri);
        const float2 ri4 = mul2(ri2, ri2);
        const float2 ri6 = mul2(ri4, ri2), ri12 = mul2(ri6, ri6), ri10 = mul2(ri6, ri4);
        const float2 rim = v2((ija & kPairHB) ? ri10.x : ri6.x, (ijb & kPairHB) ? ri10.y : ri6.y);
        const float2 km = v2((ija & kPairHB) ? 10.f : 6.f, (ijb & kPairHB) ? 10.f : 6.f);
        const float2 a12 = mul2(c12, ri12), am = mul2(cm, rim);
        const float2 elj = sub2(a12, am);
        const float2 tex = mul2(s2(kex), r);
        const float2 ex = v2(ex2_ftz(tex.x), ex2_ftz(tex.y));
        const float2 den = fma2(s2(msk), ex, s2(1.f));
        const float2 D = fma2(s2(msA), den, s2(msB));  // eps(r) = D / den
        const float2 rD = v2(rcp_ftz(D.x), rcp_ftz(D.y));
        const float2 u = mul2(ri, rD);
        const float2 cqu = mul2(cq, u);
        const float2 eel = mul2(cqu, den);
        const float2 tgs = mul2(s2(kgs), rr2);
        const float2 gs = v2(ex2_ftz(tgs.x), ex2_ftz(tgs.y));
        const float2 eds = mul2(cd, gs);
        if (GRAD) {
            // (dE/dr) / r of the three terms
            float2 dlj = mul2(fma2(km, am, mul2(s2(-12.f), a12)), ri2);
            if (elj.x > cap) dlj.x = 0.f;
            if (elj.y > cap) dlj.y = 0.f;
            // with u = 1 / (r D) and den' = -lambda k e^(-lambda r):
            // (dE_el/dr) / r = cq u / r (den' - den (A den' / D + 1 / r))
            const float2 dden = mul2(s2(-mslb * msk), ex);
            const float2 s = fma2(mul2(s2(-mslb * msk * msA), ex), rD, ri);
            const float2 deel = mul2(mul2(cqu, ri), fma2(mul2(den, s2(-1.f)), s, dden));
            const float2 cp = add2(fma2(eds, s2(-inv_s2), dlj), deel);
            const float cpa = fla ? 0.f : cp.x, cpb = flb ? 0.f : cp.y;
            ws.c[ia] = cpa;
            ws.c[ib] = cpb;
            const float coa = cpa;
            rfx = fmaf(coa, dx.x, rfx);
            rfy = fmaf(coa, dy.x, rfy);
            rfz = fmaf(coa, dz.x, rfz);
            if (ija & kPairRowEnd) {
                ws.f[(uint32_t)ija >> 24] = make_float4(rfx, rfy, rfz, 0.f);
                rfx = rfy = rfz = 0.f;
            }
            const float cob = cpb;
            rfx = fmaf(cob, dx.y, rfx);
            rfy = fmaf(cob, dy.y, rfy);
            rfz = fmaf(cob, dz.y, rfz);
            if (ijb & kPairRowEnd) {
                ws.f[(uint32_t)ijb >> 24] = make_float4(rfx, rfy, rfz, 0.f);
                rfx = rfy = rfz = 0.f;
            }
        }
        e2 = add2(e2, add2(add2(v2(fminf(elj.x, cap), fminf(elj.y, cap)), eel), eds));
    }
    e += e2.x + e2.y;
    ScoreOut out;
    out.e = warp_sum(e);
    out.gtan = 0.f;
    out.tx = out.ty = out.tz = 0.f;
    if (!GRAD) return out;
    __syncwarp();
    // force gather: f_atom += sum over its pairs that its row did not cover of
    // c_p (x_atom - x_partner), formed as x_atom sum c_p - sum c_p x_partner;
    // the atom's last group stores (sum c_p, sum c_p x_partner) in pm[atom]
    // and the scan below adds the force; every lane runs the same number of
    // groups of four entries, so consecutive groups' loads overlap
    const int ngroups = L->gsteps;
    float sc = 0.f, bx = 0.f, by = 0.f, bz = 0.f;  // sum c_p and sum c_p x_partner of the current atom
#pragma unroll 2
    for (int k = 0; k < ngroups; ++k) {
        const uint4 ge = reinterpret_cast<const uint4*>(P.gent)[k * 32 + lane];
        const uint32_t e0 = ge.x, e1 = ge.y, e2 = ge.z, e3 = ge.w;
        const float c0 = ws.c[(e0 >> 14) & 0xffff], c1 = ws.c[(e1 >> 14) & 0xffff],
                    c2 = ws.c[(e2 >> 14) & 0xffff], c3 = ws.c[(e3 >> 14) & 0xffff];
        const float4 x0 = ws.xyz[e0 & 127], x1 = ws.xyz[e1 & 127], x2 = ws.xyz[e2 & 127], x3 = ws.xyz[e3 & 127];
        sc += (c0 + c1) + (c2 + c3);
        bx = fmaf(c3, x3.x, fmaf(c2, x2.x, fmaf(c1, x1.x, fmaf(c0, x0.x, bx))));
        by = fmaf(c3, x3.y, fmaf(c2, x2.y, fmaf(c1, x1.y, fmaf(c0, x0.y, by))));
        bz = fmaf(c3, x3.z, fmaf(c2, x2.z, fmaf(c1, x1.z, fmaf(c0, x0.z, bz))));
        if (e3 >> 31) {  // the atom's last group
            ws.pm[(e0 >> 7) & 127] = make_float4(sc, bx, by, bz);
            sc = bx = by = bz = 0.f;
        }
    }
    __syncwarp();
    // Per atom: total force f and moment m = (x - t) x f.  Inclusive prefix
    // sums over the depth-first atom order go to ws.f / ws.pm; the atoms moved
    // by torsion k are the positions [lo, hi), so
    //   dE/dtheta_k = u . ((x - x_a) x f) summed there = u . M_k - (u x (x_a - t)) . F_k
    // with F_k, M_k differences of prefix sums and u the posed axis a -> b.
    // Lane l holds positions APL l + j: a running sum over its own atoms,
    // then one warp scan of the lane totals; position APL l + APL - 1 takes the
    // warp scan's value, the others the previous lanes' total plus their
    // running sum.
    const float tx = g[0], ty = g[1], tz = g[2];
    float run[APL][6];
#pragma unroll
    for (int j = 0; j < APL; ++j) {
        const int a = lane + 32 * j;
        float v0 = 0.f, v1 = 0.f, v2 = 0.f, v3 = 0.f, v4 = 0.f, v5 = 0.f;
        if (APL * lane + j < N) {
            // total force: map gradient + row sum + x sum c_p - sum c_p x_partner
            const float4 fi = ws.f[a], gi = ws.pm[a], x = ws.xyz[a];
            v0 = fxr[j] + (fi.x + fmaf(x.x, gi.x, -gi.y));
            v1 = fyr[j] + (fi.y + fmaf(x.y, gi.x, -gi.z));
            v2 = fzr[j] + (fi.z + fmaf(x.z, gi.x, -gi.w));
            const float rx = x.x - tx, ry = x.y - ty, rz = x.z - tz;
            v3 = ry * v2 - rz * v1;
            v4 = rz * v0 - rx * v2;
            v5 = rx * v1 - ry * v0;
        }
        if (j > 0) {  // two-wide adds
            const float2 a2 = __fadd2_rn(make_float2(run[j - 1][0], run[j - 1][1]), make_float2(v0, v1));
            const float2 b2 = __fadd2_rn(make_float2(run[j - 1][2], run[j - 1][3]), make_float2(v2, v3));
            const float2 d2 = __fadd2_rn(make_float2(run[j - 1][4], run[j - 1][5]), make_float2(v4, v5));
            v0 = a2.x; v1 = a2.y; v2 = b2.x; v3 = b2.y; v4 = d2.x; v5 = d2.y;
        }
        run[j][0] = v0; run[j][1] = v1; run[j][2] = v2; run[j][3] = v3; run[j][4] = v4; run[j][5] = v5;
    }
    float s0 = run[APL - 1][0], s1 = run[APL - 1][1], s2 = run[APL - 1][2], s3 = run[APL - 1][3],
          s4 = run[APL - 1][4], s5 = run[APL - 1][5];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float u0 = __shfl_up_sync(FULL_MASK, s0, o), u1 = __shfl_up_sync(FULL_MASK, s1, o),
                    u2 = __shfl_up_sync(FULL_MASK, s2, o), u3 = __shfl_up_sync(FULL_MASK, s3, o),
                    u4 = __shfl_up_sync(FULL_MASK, s4, o), u5 = __shfl_up_sync(FULL_MASK, s5, o);
        if (lane >= o) {  // two-wide adds
            const float2 a2 = __fadd2_rn(make_float2(s0, s1), make_float2(u0, u1));
            const float2 b2 = __fadd2_rn(make_float2(s2, s3), make_float2(u2, u3));
            const float2 d2 = __fadd2_rn(make_float2(s4, s5), make_float2(u4, u5));
            s0 = a2.x; s1 = a2.y; s2 = b2.x; s3 = b2.y; s4 = d2.x; s5 = d2.y;
        }
    }
    ws.f[lane + 32 * (APL - 1)] = make_float4(s0, s1, s2, 0.f);
    ws.pm[lane + 32 * (APL - 1)] = make_float4(s3, s4, s5, 0.f);
    if (APL > 1) {
        // the total of the lanes before this one
        float e0 = __shfl_up_sync(FULL_MASK, s0, 1), e1 = __shfl_up_sync(FULL_MASK, s1, 1),
              e2p = __shfl_up_sync(FULL_MASK, s2, 1), e3 = __shfl_up_sync(FULL_MASK, s3, 1),
              e4 = __shfl_up_sync(FULL_MASK, s4, 1), e5 = __shfl_up_sync(FULL_MASK, s5, 1);
        if (lane == 0) e0 = e1 = e2p = e3 = e4 = e5 = 0.f;
#pragma unroll
        for (int j = 0; j + 1 < APL; ++j) {
            const float2 a2 = __fadd2_rn(make_float2(e0, e1), make_float2(run[j][0], run[j][1]));
            const float2 b2 = __fadd2_rn(make_float2(e2p, e3), make_float2(run[j][2], run[j][3]));
            const float2 d2 = __fadd2_rn(make_float2(e4, e5), make_float2(run[j][4], run[j][5]));
            ws.f[lane + 32 * j] = make_float4(a2.x, a2.y, b2.x, 0.f);
            ws.pm[lane + 32 * j] = make_float4(b2.y, d2.x, d2.y, 0.f);
        }
    }
    __syncwarp();
    float val = 0.f;
    if (lane < 6) {
        const float4 F = ws.f[L->last_idx], Mt = ws.pm[L->last_idx];
        val = lane == 0 ? F.x : lane == 1 ? F.y : lane == 2 ? F.z : lane == 3 ? Mt.x : lane == 4 ? Mt.y : Mt.z;
    } else if (lane < 6 + T) {
        const int k = lane - 6;
        const int lo = L->lo_idx[k], hi = L->hi_idx[k];
        float4 F = ws.f[hi], Mk = ws.pm[hi];
        if (lo >= 0) {
            const float4 F0 = ws.f[lo], M0 = ws.pm[lo];
            F.x -= F0.x; F.y -= F0.y; F.z -= F0.z;
            Mk.x -= M0.x; Mk.y -= M0.y; Mk.z -= M0.z;
        }
        const float4 xa = ws.xyz[L->ta[k]], xb = ws.xyz[L->tb[k]];
        float ux = xb.x - xa.x, uy = xb.y - xa.y, uz = xb.z - xa.z;
        const float un = rsqrtf(ux * ux + uy * uy + uz * uz);
        ux *= un; uy *= un; uz *= un;
        const float ax = xa.x - tx, ay = xa.y - ty, az = xa.z - tz;
        const float gx = uy * az - uz * ay, gy = uz * ax - ux * az, gz = ux * ay - uy * ax;
        val = ux * Mk.x + uy * Mk.y + uz * Mk.z - (gx * F.x + gy * F.y + gz * F.z);
    }
    out.gtan = val;
    out.tx = __shfl_sync(FULL_MASK, val, 3);
    out.ty = __shfl_sync(FULL_MASK, val, 4);
    out.tz = __shfl_sync(FULL_MASK, val, 5);
    return out;
}

// ------------------------------------------------------------------ launch geometry
Geo make_geo(int apl, int nslots, size_t lig_bytes)
{
    Geo g;
    g.apl = apl <= 1 ? 1 : (apl >= 4 ? 4 : apl);
    g.na = 32 * g.apl;
    g.nslots = nslots < 32 ? 32 : (nslots + 31) / 32 * 32;
    g.lig_bytes = (lig_bytes + 255) / 256 * 256;
    const size_t per_warp = warp_smem_floats(g.na, g.nslots) * sizeof(float);
    // a ligand blob that leaves no room for two warps stays in global memory
    if (g.lig_bytes + 2 * per_warp > 220u * 1024u) g.lig_bytes = 0;
    // two resident blocks per SM when the ligand and at least 4 warps fit in
    // half of the 228 KB, else one block of up to 220 KB
    g.wpb = kMaxWarpsPerBlock;
    while (g.wpb > 4 && g.lig_bytes + (size_t)g.wpb * per_warp > 113u * 1024u) --g.wpb;
    if (g.lig_bytes + (size_t)g.wpb * per_warp > 113u * 1024u)
        while (g.wpb > 1 && g.lig_bytes + (size_t)g.wpb * per_warp > 220u * 1024u) --g.wpb;
    g.smem = g.lig_bytes + (size_t)g.wpb * per_warp;
    return g;
}

Geo make_geo_explicit(int apl, int nslots, size_t lig_bytes, bool staged, int wpb)
{
    Geo g = make_geo(apl, nslots, lig_bytes);
    if (!staged) g.lig_bytes = 0;
    else g.lig_bytes = (lig_bytes + 255) / 256 * 256;
    g.wpb = wpb < 1 ? 1 : (wpb > kMaxWarpsPerBlock ? kMaxWarpsPerBlock : wpb);
    g.smem = g.lig_bytes + (size_t)g.wpb * warp_smem_floats(g.na, g.nslots) * sizeof(float);
    return g;
}

template <typename K>
static cudaError_t allow_smem(K kernel, size_t bytes)
{
    if (bytes <= 48u * 1024u) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

static unsigned blocks_for(long nwarps, const Geo& g) { return (unsigned)((nwarps + g.wpb - 1) / g.wpb); }

// ------------------------------------------------------------------ score / pose API kernels
// One pose's energy and gradient into energy[0] and grad[0 ..]: the gene
// gradient (dE/dt, dE/dq by the chain rule, dE/dtheta; 7 + T values) or the
// tangent gradient (6 + T values).  gin: the pose's 7 + T genes.
template <int APL>
__device__ __forceinline__ void score_pose(const LigandRef& SL, const MapsDev& M, const WarpView& ws,
                                           const float* __restrict__ gin, float* __restrict__ energy,
                                           float* __restrict__ grad, int grad_kind, int lane, int grad_width = 0)
{
    const LigandDev* L = SL.hdr;
    const int T = L->ntors, G = 7 + T, D = 6 + T;
    if (lane < G) ws.genes[lane] = gin[lane];
    __syncwarp();
    if (grad_kind == ADG_GRAD_NONE) {
        ScoreOut o = warp_score<APL, false>(L, SL.pairs, M, ws.genes, ws, lane);
        if (lane == 0) energy[0] = o.e;
        return;
    }
    ScoreOut o = warp_score<APL, true>(L, SL.pairs, M, ws.genes, ws, lane);
    if (lane == 0) energy[0] = o.e;
    if (grad_kind == ADG_GRAD_TANGENT) {
        if (lane < max(D, grad_width)) grad[lane] = lane < D ? o.gtan : 0.f;  // a padded row's tail is 0
        return;
    }
    // gene gradient: t and theta from the tangent gradient, q by the chain rule
    // dE/dq = 2 (-tau.v, w tau + tau x v) / |q| with q/|q| = (w, v).
    const float prev = __shfl_sync(FULL_MASK, o.gtan, lane > 0 ? lane - 1 : 0);
    float val = 0.f;
    if (lane < 3) val = o.gtan;
    else if (lane < 7) {
        float qw = ws.genes[3], qx = ws.genes[4], qy = ws.genes[5], qz = ws.genes[6];
        const float qn = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz), iq = 1.f / qn;
        qw *= iq; qx *= iq; qy *= iq; qz *= iq;
        const float tx = o.tx, ty = o.ty, tz = o.tz;
        if (lane == 3) val = -2.f * (tx * qx + ty * qy + tz * qz) * iq;
        else if (lane == 4) val = 2.f * (qw * tx + (ty * qz - tz * qy)) * iq;
        else if (lane == 5) val = 2.f * (qw * ty + (tz * qx - tx * qz)) * iq;
        else val = 2.f * (qw * tz + (tx * qy - ty * qx)) * iq;
    } else if (lane < G) val = prev;
    if (lane < max(G, grad_width)) grad[lane] = lane < G ? val : 0.f;
}

template <int APL>
__global__ void __launch_bounds__(kMaxWarpsPerBlock * 32, ADG_MIN_BLOCKS) k_score(MapsDev M, LigandRef LR, int na, int nslots, int lig_bytes,
                                                                  const float* __restrict__ genes, int npose,
                                                                  float* __restrict__ energy, float* __restrict__ grad,
                                                                  int grad_kind)
{
    const int lane = threadIdx.x & 31;
    const long pose = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const LigandRef SL = stage_ligand(LR, lig_bytes);
    if (pose >= npose) return;
    const WarpView ws = warp_view(na, nslots, lig_bytes);
    const int T = SL.hdr->ntors, G = 7 + T, D = 6 + T;
    score_pose<APL>(SL, M, ws, genes + pose * G, energy + pose,
                    grad ? grad + pose * (grad_kind == ADG_GRAD_TANGENT ? D : G) : nullptr, grad_kind, lane);
}

// Poses of several ligands in one launch: block b serves ligand J.blk_lig[b]
// (the ligand's blocks are consecutive, from J.lig_blk0; J.lig_nblk of them);
// warp w of the ligand's blocks takes its poses w, w + (warps of the
// ligand), ..., rows J.lig_row0 .. of the row-strided arrays, so the
// ligand's tables staged once per block serve several poses per warp.
template <int APL>
__global__ void __launch_bounds__(kMaxWarpsPerBlock * 32, ADG_MIN_BLOCKS) k_score_multi(MapsDev M, ScoreMultiDev J, int na, int nslots,
                                                                        int lig_bytes, const float* __restrict__ genes,
                                                                        float* __restrict__ energy,
                                                                        float* __restrict__ grad, int grad_kind)
{
    const int lane = threadIdx.x & 31;
    const int lig = J.blk_lig[blockIdx.x];
    const LigandRef SL = stage_ligand(J.ligs[lig], lig_bytes);
    const int wpb = blockDim.x >> 5;
    const int stride = J.lig_nblk[lig] * wpb;
    const WarpView ws = warp_view(na, nslots, lig_bytes);
    for (int local = (blockIdx.x - J.lig_blk0[lig]) * wpb + (threadIdx.x >> 5); local < J.lig_npose[lig];
         local += stride) {
        const long row = (long)J.lig_row0[lig] + local;
        score_pose<APL>(SL, M, ws, genes + row * J.stride, energy + row, grad ? grad + row * J.stride : nullptr,
                        grad_kind, lane, J.stride);
        __syncwarp();
    }
}

cudaError_t launch_score(cudaStream_t st, const MapsDev& m, const LigandRef& l, const Geo& g, const float* genes,
                         int npose, float* energy, float* grad, int grad_kind)
{
    if (npose <= 0) return cudaSuccess;
    const unsigned blocks = blocks_for(npose, g);
    const unsigned threads = g.wpb * 32;
    cudaError_t e;
#define ADG_SCORE(A)                                                                                            \
    e = allow_smem(k_score<A>, g.smem);                                                                         \
    if (e != cudaSuccess) return e;                                                                             \
    k_score<A><<<blocks, threads, g.smem, st>>>(m, l, g.na, g.nslots, (int)g.lig_bytes, genes, npose, energy, grad, \
                                                grad_kind);
    if (g.apl == 1) { ADG_SCORE(1) }
    else if (g.apl == 2) { ADG_SCORE(2) }
    else if (g.apl == 3) { ADG_SCORE(3) }
    else { ADG_SCORE(4) }
#undef ADG_SCORE
    return cudaGetLastError();
}

cudaError_t launch_score_multi(cudaStream_t st, const MapsDev& m, const ScoreMultiDev& j, int nblocks, const Geo& g,
                               const float* genes, float* energy, float* grad, int grad_kind)
{
    if (nblocks <= 0) return cudaSuccess;
    const unsigned threads = g.wpb * 32;
    cudaError_t e;
#define ADG_SCORE_MULTI(A)                                                                                        \
    e = allow_smem(k_score_multi<A>, g.smem);                                                                     \
    if (e != cudaSuccess) return e;                                                                               \
    k_score_multi<A><<<(unsigned)nblocks, threads, g.smem, st>>>(m, j, g.na, g.nslots, (int)g.lig_bytes, genes, energy, \
                                                                 grad, grad_kind);
    if (g.apl == 1) { ADG_SCORE_MULTI(1) }
    else if (g.apl == 2) { ADG_SCORE_MULTI(2) }
    else if (g.apl == 3) { ADG_SCORE_MULTI(3) }
    else { ADG_SCORE_MULTI(4) }
#undef ADG_SCORE_MULTI
    return cudaGetLastError();
}

__global__ void __launch_bounds__(kMaxWarpsPerBlock * 32) k_pose(LigandRef LR, int na, int nslots,
                                                                 const float* __restrict__ genes, int npose,
                                                                 float* __restrict__ xyz)
{
    const int lane = threadIdx.x & 31;
    const long pose = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (pose >= npose) return;
    const WarpView ws = warp_view(na, nslots, 0);
    const LigandDev* L = LR.hdr;
    const int G = 7 + L->ntors, N = L->natoms;
    if (lane < G) ws.genes[lane] = genes[pose * G + lane];
    __syncwarp();
    warp_pose<4, true>(L, ws.genes, ws, lane);
    for (int j = 0; j < L->apl && L->apl * lane + j < N; ++j) {  // this lane's atoms
        const int a = lane + 32 * j;
        const float4 x = ws.xyz[a];
        const long o = (pose * N + L->old_of_new[a]) * 3;
        xyz[o + 0] = x.x;
        xyz[o + 1] = x.y;
        xyz[o + 2] = x.z;
    }
}

cudaError_t launch_pose(cudaStream_t st, const LigandRef& l, const Geo& g0, const float* genes, int npose, float* xyz)
{
    if (npose <= 0) return cudaSuccess;
    const Geo g = make_geo(4, g0.nslots, 0);  // k_pose indexes up to 4 atoms per lane
    cudaError_t e = allow_smem(k_pose, g.smem);
    if (e != cudaSuccess) return e;
    k_pose<<<blocks_for(npose, g), g.wpb * 32, g.smem, st>>>(l, g.na, g.nslots, genes, npose, xyz);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ moves
// Unit quaternion of the rotation vector w (angle |w| about w/|w|).
__device__ __forceinline__ float4 quat_from_rotvec(float wx, float wy, float wz)
{
    const float ang = sqrtf(wx * wx + wy * wy + wz * wz);
    if (ang < 1e-12f) return make_float4(1.f, 0.5f * wx, 0.5f * wy, 0.5f * wz);
    float s, c;
    sincosf(0.5f * ang, &s, &c);
    s /= ang;
    return make_float4(c, s * wx, s * wy, s * wz);  // (w, x, y, z)
}

// a (x) b for quaternions stored (w, x, y, z).
__device__ __forceinline__ float4 quat_mul(float4 a, float4 b)
{
    return make_float4(a.x * b.x - a.y * b.y - a.z * b.z - a.w * b.w, a.x * b.y + b.x * a.y + a.z * b.w - a.w * b.z,
                       a.x * b.z + b.x * a.z + a.w * b.y - a.y * b.w, a.x * b.w + b.x * a.w + a.y * b.z - a.z * b.y);
}

__device__ __forceinline__ float4 quat_normalise(float4 q)
{
    const float in = 1.f / sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    return make_float4(q.x * in, q.y * in, q.z * in, q.w * in);
}

// out = x (+) sign*xi, xi distributed over lanes (lane d holds tangent component d):
// t += xi_t; q <- exp(xi_w) (x) q, normalised; theta += xi_theta.
__device__ __forceinline__ void warp_step(const float* x, float* out, float xi, float sign, int T, int lane)
{
    const float w0 = __shfl_sync(FULL_MASK, xi, 3), w1 = __shfl_sync(FULL_MASK, xi, 4),
                w2 = __shfl_sync(FULL_MASK, xi, 5);
    const float prev = __shfl_sync(FULL_MASK, xi, lane > 0 ? lane - 1 : 0);
    if (lane < 3) {
        out[lane] = x[lane] + sign * xi;
    } else if (lane < 7) {
        const float4 dq = quat_from_rotvec(sign * w0, sign * w1, sign * w2);
        const float4 nq = quat_normalise(quat_mul(dq, make_float4(x[3], x[4], x[5], x[6])));
        out[lane] = lane == 3 ? nq.x : lane == 4 ? nq.y : lane == 5 ? nq.z : nq.w;
    } else if (lane < 7 + T) {
        out[lane] = x[lane] + sign * prev;
    }
    __syncwarp();
}

// Box-Muller Gaussian of tangent dimension d, Solis-Wets iteration `it`.
__device__ __forceinline__ float ls_gauss(const Rng& r, int it, int d)
{
    const uint4 w = r.block(P_LS, it * 8 + d / 4);
    const int p = (d / 2) % 2;
    const uint32_t a = p ? w.z : w.x, b = p ? w.w : w.y;
    const float u1 = u01_open0(a), u2 = u01(b);
    const float rad = sqrtf(-2.f * logf(u1));
    float s, c;
    sincospif(2.f * u2, &s, &c);
    return (d & 1) ? rad * s : rad * c;
}

// Solis & Wets (1981) adaptive random search on the genotype in ws.genes.
template <int APL>
__device__ __forceinline__ int warp_solis_wets(const LigandDev* L, const PairsDev& P, const MapsDev& M,
                                               const SearchDev& S, const Rng& rng, const WarpView& ws, float& e,
                                               int lane)
{
    const int T = L->ntors, D = 6 + T;
    const float scale = lane < 3 ? S.sw_scale_t : (lane < 6 ? S.sw_scale_rot : S.sw_scale_tors);
    float bias = 0.f, rho = S.sw_rho0;
    int succ = 0, fail = 0, nev = 0;
    for (int it = 0; it < S.ls_max_iters && rho >= S.sw_rho_min; ++it) {
        const float xi = lane < D ? bias + rho * scale * ls_gauss(rng, it, lane) : 0.f;
        warp_step(ws.genes, ws.cand, xi, 1.f, T, lane);
        const float e1 = warp_score<APL, false>(L, P, M, ws.cand, ws, lane).e;
        ++nev;
        if (e1 < e) {
            if (lane < 7 + T) ws.genes[lane] = ws.cand[lane];
            e = e1;
            bias = 0.4f * xi + 0.2f * bias;
            ++succ;
            fail = 0;
        } else {
            warp_step(ws.genes, ws.cand, xi, -1.f, T, lane);
            const float e2 = warp_score<APL, false>(L, P, M, ws.cand, ws, lane).e;
            ++nev;
            if (e2 < e) {
                if (lane < 7 + T) ws.genes[lane] = ws.cand[lane];
                e = e2;
                bias = bias - 0.4f * xi;
                ++succ;
                fail = 0;
            } else {
                bias *= 0.5f;
                ++fail;
                succ = 0;
            }
        }
        __syncwarp();
        if (succ >= S.sw_succ) { rho *= S.sw_expand; succ = 0; }
        if (fail >= S.sw_fail) { rho *= S.sw_contract; fail = 0; }
    }
    return nev;
}

// ADADELTA (Zeiler 2012) in the tangent space; keeps the best genotype seen.
template <int APL>
__device__ __forceinline__ int warp_adadelta(const LigandDev* L, const PairsDev& P, const MapsDev& M,
                                             const SearchDev& S, const WarpView& ws, float& e, int lane)
{
    const int T = L->ntors, G = 7 + T;
    float eg2 = 0.f, edx2 = 0.f, ebest = e;
    if (lane < G) ws.best[lane] = ws.genes[lane];
    __syncwarp();
    for (int it = 0; it < S.ls_max_iters; ++it) {
        const ScoreOut o = warp_score<APL, true>(L, P, M, ws.genes, ws, lane);
        if (o.e < ebest) {
            ebest = o.e;
            if (lane < G) ws.best[lane] = ws.genes[lane];
        }
        const float gd = o.gtan;
        eg2 = S.ad_rho * eg2 + (1.f - S.ad_rho) * gd * gd;
        const float dx = -sqrtf(edx2 + S.ad_eps) / sqrtf(eg2 + S.ad_eps) * gd;
        edx2 = S.ad_rho * edx2 + (1.f - S.ad_rho) * dx * dx;
        warp_step(ws.genes, ws.cand, dx, 1.f, T, lane);
        if (lane < G) ws.genes[lane] = ws.cand[lane];
        __syncwarp();
    }
    if (lane < G) ws.genes[lane] = ws.best[lane];
    __syncwarp();
    e = ebest;
    return S.ls_max_iters;
}

// ------------------------------------------------------------------ LGA kernels
__device__ __forceinline__ void warp_argmin(float& v, int& i)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const float ov = __shfl_xor_sync(FULL_MASK, v, o);
        const int oi = __shfl_xor_sync(FULL_MASK, i, o);
        if (ov < v || (ov == v && oi < i)) {
            v = ov;
            i = oi;
        }
    }
}

__device__ __forceinline__ int tournament(const float* Pe, int pop, uint32_t wa, uint32_t wb, uint32_t wwin, uint32_t thr,
                                          int& a, int& b)
{
    a = uindex(wa, pop);
    b = uindex(wb, pop);
    const float ea = Pe[a], eb = Pe[b];
    int better, worse;
    if (ea < eb || (ea == eb && a <= b)) { better = a; worse = b; }
    else { better = b; worse = a; }
    return ptest(wwin, thr) ? better : worse;
}

// Generation 0: random genotypes (t uniform in the box, q uniform on S^3 by
// Shoemake's three uniforms, theta uniform in [-pi, pi)), evaluated.
template <int APL>
__global__ void __launch_bounds__(kMaxWarpsPerBlock * 32, ADG_MIN_BLOCKS) k_dock_init(MapsDev M, SearchDev S, DockDev Dk, int na,
                                                                      int nslots, int lig_bytes, int wpl)
{
    const int lane = threadIdx.x & 31;
    // warps of one ligand are padded to whole blocks (wpl per ligand), so a block has one ligand
    const long gw = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lig = (int)(gw / wpl);
    const int local = (int)(gw % wpl);
    const LigandRef LR = stage_ligand(Dk.ligs[lig], lig_bytes);
    if (local >= S.nrun * S.pop) return;
    const WarpView ws = warp_view(na, nslots, lig_bytes);
    const int run = local / S.pop, ind = local % S.pop;
    const int run_g = lig * S.nrun + run;
    const LigandDev* L = LR.hdr;
    const int T = L->ntors, G = 7 + T;
    const Rng rng{S.key0, S.key1, Dk.lig_id[lig], (uint32_t)(Dk.run0 + run), (uint32_t)ind, 0u};
    float v = 0.f;
    if (lane < 3) {
        const uint4 wd = rng.block(P_INIT, 0);
        const float lo = lane == 0 ? M.ox : lane == 1 ? M.oy : M.oz;
        const float hi = lane == 0 ? M.hx : lane == 1 ? M.hy : M.hz;
        v = lo + u01(word(wd, lane)) * (hi - lo);
    } else if (lane < 7) {
        const uint4 wd = rng.block(P_INIT, 1);
        const float u1 = u01(wd.x), u2 = u01(wd.y), u3 = u01(wd.z);
        const float s1 = sqrtf(1.f - u1), s2 = sqrtf(u1);
        float sa, ca, sb, cb;
        sincospif(2.f * u2, &sa, &ca);
        sincospif(2.f * u3, &sb, &cb);
        v = lane == 3 ? s2 * cb : lane == 4 ? s1 * sa : lane == 5 ? s1 * ca : s2 * sb;
    } else if (lane < G) {
        const int k = lane - 7;
        const uint4 wd = rng.block(P_INIT, 2 + k / 4);
        v = -3.14159265358979f + 6.28318530717959f * u01(word(wd, k % 4));
    }
    if (lane < G) ws.genes[lane] = v;
    __syncwarp();
    const float e = warp_score<APL, false>(L, LR.pairs, M, ws.genes, ws, lane).e;
    float* pg = Dk.pop_genes[0] + ((long)run_g * S.pop + ind) * kGeneStride;
    if (lane < G) pg[lane] = v;
    if (lane == 0) {
        Dk.pop_e[0][(long)run_g * S.pop + ind] = e;
        atomicAdd(&Dk.evals[run_g], 1ull);
    }
}

// One GA generation of one individual per warp: selection, crossover,
// mutation, offspring evaluation, local search.  Per-generation evaluation
// counts accumulate in evals[nruns + run] until k_dock_bookkeep folds them
// in, so every warp of a generation sees the same total when it decides
// whether its run is still active.
template <int APL, int LS, bool STAGED>
__global__ void __launch_bounds__(kMaxWarpsPerBlock * 32, ADG_MIN_BLOCKS) k_dock_generation(MapsDev M, SearchDev S, DockDev Dk,
                                                                            int na, int nslots, int lig_bytes, int wpl,
                                                                            int gen_arg, const int* __restrict__ gen_dev)
{
    const int lane = threadIdx.x & 31;
    // inside a graph loop the device counter holds the generations completed so far
    const int gen = gen_dev ? *gen_dev + 1 : gen_arg;
    // warps of one ligand are padded to whole blocks (wpl per ligand), so a block has one ligand
    const long gw = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long nruns = (long)Dk.nlig * S.nrun;
    const int lig = (int)(gw / wpl);
    const int local = (int)(gw % wpl);
    const LigandRef LR = stage_ligand<STAGED ? 1 : 0>(Dk.ligs[lig], lig_bytes);
    if (local >= S.nrun * S.pop) return;
    const int run = local / S.pop, ind = local % S.pop;
    const int run_g = lig * S.nrun + run;
    if (Dk.evals[run_g] >= (unsigned long long)S.nev || gen > S.max_gen || Dk.stopped[run_g]) return;
    const WarpView ws = warp_view(na, nslots, lig_bytes);
    const LigandDev* L = LR.hdr;
    const int T = L->ntors, G = 7 + T, nb = 2 + T, pop = S.pop;
    const Rng rng{S.key0, S.key1, Dk.lig_id[lig], (uint32_t)(Dk.run0 + run), (uint32_t)ind, (uint32_t)gen};
    const float* Pg = Dk.pop_genes[(gen - 1) & 1] + (long)run_g * pop * kGeneStride;
    const float* Pe = Dk.pop_e[(gen - 1) & 1] + (long)run_g * pop;

    // elite = argmin of the previous population (ties to the lower index)
    float bv = INFINITY;
    int bi = 0x7fffffff;
    for (int i = lane; i < pop; i += 32) {
        const float v = Pe[i];
        if (v < bv) { bv = v; bi = i; }
    }
    warp_argmin(bv, bi);
    if (bi >= pop) bi = 0;  // only when every energy is NaN

    float child = 0.f, e;
    int p1, p2, lo = -1, hi = -1, mmask = 0, nev = 0;
    int a1 = -1, b1 = -1, a2 = -1, b2 = -1;
    if (ind < S.elitism) {
        p1 = p2 = bi;
        if (lane < G) child = Pg[(long)bi * kGeneStride + lane];
        e = bv;
        if (lane < G) ws.genes[lane] = child;
        __syncwarp();
    } else {
        const uint4 w0 = rng.block(P_SELECT, 0), w1 = rng.block(P_SELECT, 1), w2 = rng.block(P_SELECT, 2);
        p1 = tournament(Pe, pop, w0.x, w0.y, w0.z, S.thr_tour, a1, b1);
        p2 = tournament(Pe, pop, w1.x, w1.y, w1.z, S.thr_tour, a2, b2);
        if (ptest(w2.x, S.thr_cross)) {
            const int c1 = uindex(w2.y, nb + 1), c2 = uindex(w2.z, nb + 1);
            lo = min(c1, c2);
            hi = max(c1, c2);
        }
        const int b = lane < 3 ? 0 : (lane < 7 ? 1 : 2 + (lane - 7));
        const int src = (b >= lo && b < hi) ? p2 : p1;
        if (lane < G) child = Pg[(long)src * kGeneStride + lane];
        bool mut = false;
        if (lane < G) mut = ptest(word(rng.block(P_SELECT, 3 + b / 4), b % 4), S.thr_mut);
        const bool first = lane == 0 || lane == 3 || (lane >= 7 && lane < G);
        const unsigned bal = __ballot_sync(FULL_MASK, mut && first);
        mmask = (int)((bal & 1u) | (((bal >> 3) & 1u) << 1) | ((bal >> 7) << 2));
        if (mut && lane < 3) child += S.mut_t * (2.f * u01(word(rng.block(P_MUTATE, 0), lane)) - 1.f);
        if (mut && lane >= 7 && lane < G) child += S.mut_tors * (2.f * u01(rng.block(P_MUTATE, b).x) - 1.f);
        const float q0 = __shfl_sync(FULL_MASK, child, 3), q1 = __shfl_sync(FULL_MASK, child, 4),
                    q2 = __shfl_sync(FULL_MASK, child, 5), q3 = __shfl_sync(FULL_MASK, child, 6);
        if ((mmask & 2) && lane >= 3 && lane < 7) {
            const uint4 wm = rng.block(P_MUTATE, 1);
            const float z = 2.f * u01(wm.x) - 1.f;
            float sp, cp;
            sincospif(2.f * u01(wm.y), &sp, &cp);
            const float s = sqrtf(1.f - z * z);
            const float ang = S.mut_rot * (2.f * u01(wm.z) - 1.f);
            const float4 dq = quat_from_rotvec(ang * s * cp, ang * s * sp, ang * z);
            const float4 nq = quat_normalise(quat_mul(dq, make_float4(q0, q1, q2, q3)));
            child = lane == 3 ? nq.x : lane == 4 ? nq.y : lane == 5 ? nq.z : nq.w;
        }
        if (lane < G) ws.genes[lane] = child;
        __syncwarp();
        e = warp_score<APL, false>(L, LR.pairs, M, ws.genes, ws, lane).e;
        nev = 1;
    }
    // local search on this individual with probability ls_rate (Lamarckian write-back)
    const bool ls_applied = LS != ADG_LS_NONE && ptest(rng.block(P_LSPICK, 0).x, S.thr_ls);
    // the decision record is written before the local search, so none of its
    // fields stays live across it
    const bool traced = Dk.trace_ngen > 0 && gen <= Dk.trace_ngen && lig == 0;
    const long slot = ((long)run * Dk.trace_ngen + (gen - 1)) * pop + ind;
    if (traced && lane == 0) {
        int* d = Dk.tr_dec + slot * ADG_TRACE_WIDTH;
        d[0] = p1; d[1] = p2; d[2] = lo; d[3] = hi; d[4] = mmask; d[5] = ls_applied ? 1 : 0;
        d[6] = a1; d[7] = b1; d[8] = a2; d[9] = b2; d[10] = 0; d[11] = 0;
    }
    if (ls_applied) {
        if (LS == ADG_LS_SOLIS_WETS) nev += warp_solis_wets<APL>(L, LR.pairs, M, S, rng, ws, e, lane);
        else nev += warp_adadelta<APL>(L, LR.pairs, M, S, ws, e, lane);
    }
    float* Ng = Dk.pop_genes[gen & 1] + ((long)run_g * pop + ind) * kGeneStride;
    if (lane < G) Ng[lane] = ws.genes[lane];
    if (lane == 0) {
        Dk.pop_e[gen & 1][(long)run_g * pop + ind] = e;
        atomicAdd(&Dk.evals[nruns + run_g], (unsigned long long)nev);
    }
    if (traced) {
        if (lane == 0) Dk.tr_e[slot] = e;
        if (lane < G) Dk.tr_genes[slot * kGeneStride + lane] = ws.genes[lane];
    }
}

// One thread per run: fold the generation's evaluations into the total,
// record the last completed generation and the run's best energy, apply
// autostop (paper Sec. 1.1: population standard deviation of the best energy
// over the last 10 generations below stopstd), count runs active for gen+1.
__global__ void k_dock_bookkeep(SearchDev S, DockDev Dk, int gen_arg, const int* __restrict__ gen_dev, int* active)
{
    const int gen = gen_dev ? *gen_dev + 1 : gen_arg;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int nruns = Dk.nlig * S.nrun;
    if (r >= nruns) return;
    const unsigned long long nev = (unsigned long long)S.nev;
    if (Dk.evals[r] < nev && gen <= S.max_gen && !Dk.stopped[r]) {
        Dk.evals[r] += Dk.evals[nruns + r];
        Dk.evals[nruns + r] = 0ull;
        Dk.gen_done[r] = gen;
        const float* Pe = Dk.pop_e[gen & 1] + (long)r * S.pop;
        float b = Pe[0];
        for (int i = 1; i < S.pop; ++i) b = fminf(b, Pe[i]);
        float* h = Dk.best_hist + 10 * r;
        h[(gen - 1) % 10] = b;
        if (gen <= Dk.best_trace_len) Dk.best_trace[(long)r * Dk.best_trace_len + gen - 1] = b;
        if (S.autostop && gen >= 10) {
            float m = 0.f, v = 0.f;
            for (int k = 0; k < 10; ++k) m += h[k];
            m *= 0.1f;
            for (int k = 0; k < 10; ++k) v += (h[k] - m) * (h[k] - m);
            if (sqrtf(0.1f * v) < S.stopstd) Dk.stopped[r] = 1;
        }
    }
    if (Dk.evals[r] < nev && gen + 1 <= S.max_gen && !Dk.stopped[r]) atomicAdd(active, 1);
}

// Warps per ligand: its nrun * pop individuals padded to whole blocks.
static int warps_per_ligand(const SearchDev& s, const Geo& g) { return (s.nrun * s.pop + g.wpb - 1) / g.wpb * g.wpb; }

cudaError_t launch_dock_init(cudaStream_t st, const MapsDev& m, const SearchDev& s, const DockDev& d, const Geo& g)
{
    const int wpl = warps_per_ligand(s, g);
    const unsigned blocks = (unsigned)((long)d.nlig * wpl / g.wpb), threads = g.wpb * 32;
    cudaError_t e;
#define ADG_INIT(A)                                                                      \
    e = allow_smem(k_dock_init<A>, g.smem);                                              \
    if (e != cudaSuccess) return e;                                                      \
    k_dock_init<A><<<blocks, threads, g.smem, st>>>(m, s, d, g.na, g.nslots, (int)g.lig_bytes, wpl);
    if (g.apl == 1) { ADG_INIT(1) }
    else if (g.apl == 2) { ADG_INIT(2) }
    else if (g.apl == 3) { ADG_INIT(3) }
    else { ADG_INIT(4) }
#undef ADG_INIT
    return cudaGetLastError();
}

template <int APL, int LS, bool STAGED>
static cudaError_t gen_launch_form(cudaStream_t st, const MapsDev& m, const SearchDev& s, const DockDev& d,
                                   const Geo& g, int gen, const int* gen_dev)
{
    const int wpl = warps_per_ligand(s, g);
    const unsigned blocks = (unsigned)((long)d.nlig * wpl / g.wpb);
    cudaError_t e = allow_smem(k_dock_generation<APL, LS, STAGED>, g.smem);
    if (e != cudaSuccess) return e;
    k_dock_generation<APL, LS, STAGED><<<blocks, g.wpb * 32, g.smem, st>>>(m, s, d, g.na, g.nslots, (int)g.lig_bytes,
                                                                           wpl, gen, gen_dev);
    return cudaGetLastError();
}

template <int APL, int LS>
static cudaError_t gen_launch(cudaStream_t st, const MapsDev& m, const SearchDev& s, const DockDev& d, const Geo& g,
                              int gen, const int* gen_dev)
{
    return g.lig_bytes > 0 ? gen_launch_form<APL, LS, true>(st, m, s, d, g, gen, gen_dev)
                           : gen_launch_form<APL, LS, false>(st, m, s, d, g, gen, gen_dev);
}

cudaError_t launch_dock_generation(cudaStream_t st, const MapsDev& m, const SearchDev& s, const DockDev& d, const Geo& g,
                                   int gen, const int* gen_dev)
{
#define ADG_GEN(A)                                                                                               \
    if (s.ls_method == ADG_LS_SOLIS_WETS) return gen_launch<A, ADG_LS_SOLIS_WETS>(st, m, s, d, g, gen, gen_dev); \
    if (s.ls_method == ADG_LS_ADADELTA) return gen_launch<A, ADG_LS_ADADELTA>(st, m, s, d, g, gen, gen_dev);     \
    return gen_launch<A, ADG_LS_NONE>(st, m, s, d, g, gen, gen_dev);
    if (g.apl == 1) { ADG_GEN(1) }
    if (g.apl == 2) { ADG_GEN(2) }
    if (g.apl == 3) { ADG_GEN(3) }
    ADG_GEN(4)
#undef ADG_GEN
}

// ------------------------------------------------------------------ launch-geometry tuning
template <int APL, int LS, bool STAGED>
static int blocks_per_sm_form(const Geo& g)
{
    int optin = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
    if (g.smem > (size_t)optin) return 0;
    if (allow_smem(k_dock_generation<APL, LS, STAGED>, g.smem) != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_dock_generation<APL, LS, STAGED>, g.wpb * 32, g.smem) !=
        cudaSuccess)
        return 0;
    return nb;
}

template <int APL, int LS>
static int blocks_per_sm(const Geo& g)
{
    return g.lig_bytes > 0 ? blocks_per_sm_form<APL, LS, true>(g) : blocks_per_sm_form<APL, LS, false>(g);
}

int geo_blocks_per_sm(const Geo& g, int ls)
{
#define ADG_BPS(A)                                                                              \
    if (ls == ADG_LS_SOLIS_WETS) return blocks_per_sm<A, ADG_LS_SOLIS_WETS>(g);                \
    if (ls == ADG_LS_ADADELTA) return blocks_per_sm<A, ADG_LS_ADADELTA>(g);                    \
    return blocks_per_sm<A, ADG_LS_NONE>(g);
    if (g.apl == 1) { ADG_BPS(1) }
    if (g.apl == 2) { ADG_BPS(2) }
    if (g.apl == 3) { ADG_BPS(3) }
    ADG_BPS(4)
#undef ADG_BPS
}

int geo_best(int apl, int nslots, size_t lig_bytes, bool staged, int ls, Geo* out)
{
    int best_res = 0;
    for (int wpb = kMaxWarpsPerBlock; wpb >= 1; --wpb) {  // ties keep the larger block (fewer ligand copies)
        const Geo g = make_geo_explicit(apl, nslots, lig_bytes, staged, wpb);
        const int res = geo_blocks_per_sm(g, ls) * wpb;
        if (res > best_res) {
            *out = g;
            best_res = res;
        }
    }
    return best_res;
}

int geo_candidates(int apl, int nslots, size_t lig_bytes, int ls, Geo* out, int cap)
{
    int n = 0;
    for (int staged = 1; staged >= 0; --staged) {
        if (staged && lig_bytes == 0) continue;
        Geo g;
        if (geo_best(apl, nslots, lig_bytes, staged != 0, ls, &g) > 0 && n < cap) out[n++] = g;
    }
    return n;
}

// Random poses about the box centre: t = centre + U(-spread, spread) per axis,
// q uniform on S^3 (three uniforms, Shoemake), theta uniform in [-pi, pi).
__global__ void k_probe_genes(MapsDev M, int T, int npose, float spread, uint32_t seed, float* __restrict__ genes)
{
    const int pose = blockIdx.x * blockDim.x + threadIdx.x;
    if (pose >= npose) return;
    const int G = 7 + T;
    float* g = genes + (long)pose * G;
    const uint4 a = philox(make_uint4((uint32_t)pose, 0u, 0u, 7u << 20), seed, 0x7475u);
    const uint4 b = philox(make_uint4((uint32_t)pose, 1u, 0u, 7u << 20), seed, 0x7475u);
    g[0] = 0.5f * (M.ox + M.hx) + spread * (2.f * u01(a.x) - 1.f);
    g[1] = 0.5f * (M.oy + M.hy) + spread * (2.f * u01(a.y) - 1.f);
    g[2] = 0.5f * (M.oz + M.hz) + spread * (2.f * u01(a.z) - 1.f);
    const float u1 = u01(b.x), s1 = sqrtf(1.f - u1), s2 = sqrtf(u1);
    float sa, ca, sb, cb;
    sincospif(2.f * u01(b.y), &sa, &ca);
    sincospif(2.f * u01(b.z), &sb, &cb);
    g[3] = s2 * cb;
    g[4] = s1 * sa;
    g[5] = s1 * ca;
    g[6] = s2 * sb;
    for (int k = 0; k < T; k += 4) {
        const uint4 w = philox(make_uint4((uint32_t)pose, 2u + (uint32_t)k, 0u, 7u << 20), seed, 0x7475u);
        for (int i = 0; i < 4 && k + i < T; ++i) g[7 + k + i] = -3.14159265f + 6.28318531f * u01(word(w, i));
    }
}

cudaError_t launch_probe_genes(cudaStream_t st, const MapsDev& m, int T, int npose, float spread, uint32_t seed,
                               float* genes)
{
    if (npose <= 0) return cudaSuccess;
    k_probe_genes<<<(unsigned)((npose + 127) / 128), 128, 0, st>>>(m, T, npose, spread, seed, genes);
    return cudaGetLastError();
}

template <int APL, bool GRAD>
__global__ void __launch_bounds__(kMaxWarpsPerBlock * 32, ADG_MIN_BLOCKS) k_tune(MapsDev M, LigandRef LR, int na,
                                                                                int nslots, int lig_bytes,
                                                                                const float* __restrict__ genes,
                                                                                int npose, int reps,
                                                                                float* __restrict__ energy)
{
    const int lane = threadIdx.x & 31;
    const long pose = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const LigandRef SL = stage_ligand(LR, lig_bytes);
    if (pose >= npose) return;
    const WarpView ws = warp_view(na, nslots, lig_bytes);
    const LigandDev* L = SL.hdr;
    const int G = 7 + L->ntors;
    const float g0 = lane < G ? genes[pose * G + lane] : 0.f;
    float acc = 0.f;
    for (int r = 0; r < reps; ++r) {
        if (lane < G) ws.genes[lane] = lane >= 7 ? g0 + 1e-3f * (float)r : g0;
        __syncwarp();
        const ScoreOut o = warp_score<APL, GRAD>(L, SL.pairs, M, ws.genes, ws, lane);
        acc = o.e + (GRAD ? 1e-30f * __shfl_sync(FULL_MASK, o.gtan, 6) : 0.f);
        __syncwarp();
    }
    if (lane == 0) energy[pose] = acc;
}

cudaError_t launch_tune(cudaStream_t st, const MapsDev& m, const LigandRef& l, const Geo& g, const float* genes,
                        int npose, int reps, int grad, float* energy)
{
    if (npose <= 0) return cudaSuccess;
    const unsigned blocks = blocks_for(npose, g);
    const unsigned threads = g.wpb * 32;
    cudaError_t e;
#define ADG_TUNE(A, GR)                                                                                    \
    e = allow_smem(k_tune<A, GR>, g.smem);                                                                 \
    if (e != cudaSuccess) return e;                                                                        \
    k_tune<A, GR><<<blocks, threads, g.smem, st>>>(m, l, g.na, g.nslots, (int)g.lig_bytes, genes, npose, reps, \
                                                   energy);
    if (grad) {
        if (g.apl == 1) { ADG_TUNE(1, true) }
        else if (g.apl == 2) { ADG_TUNE(2, true) }
        else if (g.apl == 3) { ADG_TUNE(3, true) }
        else { ADG_TUNE(4, true) }
    } else {
        if (g.apl == 1) { ADG_TUNE(1, false) }
        else if (g.apl == 2) { ADG_TUNE(2, false) }
        else if (g.apl == 3) { ADG_TUNE(3, false) }
        else { ADG_TUNE(4, false) }
    }
#undef ADG_TUNE
    return cudaGetLastError();
}

cudaError_t launch_dock_count_active(cudaStream_t st, const SearchDev& s, const DockDev& d, int gen, int* active,
                                     const int* gen_dev)
{
    const int nruns = d.nlig * s.nrun;
    k_dock_bookkeep<<<(nruns + 127) / 128, 128, 0, st>>>(s, d, gen, gen_dev, active);
    return cudaGetLastError();
}

// Loop control of a graph-resident generation loop: continue while some run
// is active, count the completed generation, clear the active count.
__global__ void k_dock_loop_ctl(cudaGraphConditionalHandle h, int* gen_dev, int* active)
{
    const int more = *active > 0;
    *gen_dev += 1;
    *active = 0;
    cudaGraphSetConditional(h, more ? 1u : 0u);
}

cudaError_t launch_dock_loop_ctl(cudaStream_t st, cudaGraphConditionalHandle h, int* gen_dev, int* active)
{
    k_dock_loop_ctl<<<1, 1, 0, st>>>(h, gen_dev, active);
    return cudaGetLastError();
}

// Per run: best genotype of the final population and its posed coordinates.
__global__ void __launch_bounds__(kMaxWarpsPerBlock * 32) k_dock_finalize(MapsDev M, SearchDev S, DockDev Dk, int na,
                                                                          int nslots, ResultDev* __restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int run_g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nruns = Dk.nlig * S.nrun;
    if (run_g >= nruns) return;
    const WarpView ws = warp_view(na, nslots, 0);
    const int lig = run_g / S.nrun;
    const LigandDev* L = Dk.ligs[lig].hdr;
    const int G = 7 + L->ntors, N = L->natoms, gd = Dk.gen_done[run_g];
    const float* Pg = Dk.pop_genes[gd & 1] + (long)run_g * S.pop * kGeneStride;
    const float* Pe = Dk.pop_e[gd & 1] + (long)run_g * S.pop;
    float bv = INFINITY;
    int bi = 0x7fffffff;
    for (int i = lane; i < S.pop; i += 32) {
        const float v = Pe[i];
        if (v < bv) { bv = v; bi = i; }
    }
    warp_argmin(bv, bi);
    if (bi >= S.pop) bi = 0;  // only when every energy is NaN
    if (lane < G) ws.genes[lane] = Pg[(long)bi * kGeneStride + lane];
    __syncwarp();
    warp_pose<4, true>(L, ws.genes, ws, lane);
    ResultDev& R = out[run_g];
    if (lane == 0) {
        R.best_energy = bv;
        R.generations = gd;
        R.evals = (long long)Dk.evals[run_g];
    }
    if (lane < kGeneStride) R.genes[lane] = lane < G ? ws.genes[lane] : 0.f;
    for (int j = 0; j < L->apl && L->apl * lane + j < N; ++j) {  // this lane's atoms
        const int a = lane + 32 * j;
        const float4 x = ws.xyz[a];
        const int o = 3 * L->old_of_new[a];
        R.xyz[o] = x.x;
        R.xyz[o + 1] = x.y;
        R.xyz[o + 2] = x.z;
    }
}

cudaError_t launch_dock_finalize(cudaStream_t st, const MapsDev& m, const SearchDev& s, const DockDev& d, const Geo& g0,
                                 ResultDev* out)
{
    const int nruns = d.nlig * s.nrun;
    const Geo g = make_geo(4, g0.nslots, 0);  // the final pose indexes up to 4 atoms per lane
    cudaError_t e = allow_smem(k_dock_finalize, g.smem);
    if (e != cudaSuccess) return e;
    k_dock_finalize<<<blocks_for(nruns, g), g.wpb * 32, g.smem, st>>>(m, s, d, g.na, g.nslots, out);
    return cudaGetLastError();
}

// Per run: the best genotype of the final population and its pose, written
// straight into adg_result records (used where the library stages nothing
// on the host).
__global__ void __launch_bounds__(kMaxWarpsPerBlock * 32) k_dock_finalize_abi(MapsDev M, SearchDev S, DockDev Dk,
                                                                              int na, int nslots,
                                                                              adg_result* __restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int run_g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nruns = Dk.nlig * S.nrun;
    if (run_g >= nruns) return;
    const WarpView ws = warp_view(na, nslots, 0);
    const int lig = run_g / S.nrun;
    const LigandDev* L = Dk.ligs[lig].hdr;
    const int G = 7 + L->ntors, N = L->natoms, gd = Dk.gen_done[run_g];
    const float* Pg = Dk.pop_genes[gd & 1] + (long)run_g * S.pop * kGeneStride;
    const float* Pe = Dk.pop_e[gd & 1] + (long)run_g * S.pop;
    float bv = INFINITY;
    int bi = 0x7fffffff;
    for (int i = lane; i < S.pop; i += 32) {
        const float v = Pe[i];
        if (v < bv) { bv = v; bi = i; }
    }
    warp_argmin(bv, bi);
    if (bi >= S.pop) bi = 0;  // only when every energy is NaN
    if (lane < G) ws.genes[lane] = Pg[(long)bi * kGeneStride + lane];
    __syncwarp();
    warp_pose<4, true>(L, ws.genes, ws, lane);
    adg_result& R = out[run_g];
    if (lane == 0) {
        R.best_energy = bv;
        R.generations = gd;
        R.evals = (int64_t)Dk.evals[run_g];
    }
    if (lane < ADG_MAX_GENES) R.genes[lane] = lane < G ? ws.genes[lane] : 0.f;
    for (int k = lane; k < 3 * ADG_MAX_ATOMS; k += 32) R.xyz[k] = 0.f;
    __syncwarp();
    for (int j = 0; j < L->apl && L->apl * lane + j < N; ++j) {  // this lane's atoms
        const int a = lane + 32 * j;
        const float4 x = ws.xyz[a];
        const int o = 3 * L->old_of_new[a];
        R.xyz[o] = x.x;
        R.xyz[o + 1] = x.y;
        R.xyz[o + 2] = x.z;
    }
}

cudaError_t launch_dock_finalize_abi(cudaStream_t st, const MapsDev& m, const SearchDev& s, const DockDev& d,
                                     const Geo& g0, adg_result* out)
{
    const int nruns = d.nlig * s.nrun;
    const Geo g = make_geo(4, g0.nslots, 0);
    cudaError_t e = allow_smem(k_dock_finalize_abi, g.smem);
    if (e != cudaSuccess) return e;
    k_dock_finalize_abi<<<blocks_for(nruns, g), g.wpb * 32, g.smem, st>>>(m, s, d, g.na, g.nslots, out);
    return cudaGetLastError();
}

}  // namespace adg
