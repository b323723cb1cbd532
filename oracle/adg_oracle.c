/*
 * adg_oracle.c -- plain, slow FP64 CPU oracle for the AutoDock-GPU-style
 * docking hot path (arXiv 2007.03678, Sec. 1 and 1.1).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this file; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code with the CUDA path.
 *
 * The paper names the method but prints no formulas: the AutoDock4 energy
 * with vdW, hydrogen-bond, electrostatic and desolvation terms (Sec. 1), the
 * Lamarckian GA whose locally refined pose feeds crossover (Sec. 1), the
 * Solis-Wets local search (Sec. 1, Solis & Wets 1981) and the ADADELTA local
 * search (Sec. 1.1, Zeiler 2012), run `nrun` times with an evaluation budget
 * `nev` (Sec. 1.1).  Every function below states the definition it follows;
 * where the paper is silent the reading is stated in the comment.
 *
 * Everything is double precision and written for clarity: no blocking, no
 * fusion, no reordering beyond what the definitions state.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_NTYPES 7
#define ORC_NMAPS 9
#define ORC_MAP_ELEC 7
#define ORC_MAP_DESOLV 8
#define ORC_TYPE_HD 5
#define ORC_MAXATOMS 128
#define ORC_MAXTORS 16
#define ORC_MAXGENES (7 + ORC_MAXTORS)
#define ORC_MAXPAIRS (ORC_MAXATOMS * (ORC_MAXATOMS - 1) / 2)

static const double ORC_PI = 3.14159265358979323846;

/* ------------------------------------------------------------------------ */
/* Force-field table (all doubles so the Python side can fill it plainly).  */
/* ------------------------------------------------------------------------ */
typedef struct {
    double Rii[ORC_NTYPES], epsii[ORC_NTYPES], vol[ORC_NTYPES], solpar[ORC_NTYPES];
    double hb_donor[ORC_NTYPES], hb_acceptor[ORC_NTYPES], hb_R[ORC_NTYPES], hb_eps[ORC_NTYPES];
    double w_vdw, w_hb, w_elec, w_desolv, w_tors;
    double qasp, sigma, coulomb;
    double ms_A, ms_eps0, ms_lambda, ms_k;
    double r_min, e_cap, map_r_on, map_r_off, k_out;
} orc_ff;

typedef struct {
    int n[3];
    double origin[3];
    double spacing;
} orc_grid;

/* ======================================================================== */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11, */
/* "Parallel random numbers: as easy as 1, 2, 3").  Written from the        */
/* published round function: two 32x32->64 multiplies per round, key bumped */
/* by the Weyl constants between rounds, 10 rounds.                         */
/* ======================================================================== */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        uint64_t p0 = (uint64_t)PHILOX_M0 * c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Batch form used by the tests: n counters (4 words each) -> 4n words. */
void orc_philox_batch(const uint32_t* ctr, int n, uint32_t key0, uint32_t key1, uint32_t* out)
{
    uint32_t key[2] = {key0, key1};
    for (int i = 0; i < n; ++i) orc_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

/* Stream layout (reading; the paper gives no RNG): key = 64-bit seed,
 * counter = (ligand, run<<16 | individual, generation, purpose<<20 | block).
 * A draw therefore does not depend on which thread makes it. */
enum { PURPOSE_INIT = 1, PURPOSE_SELECT = 2, PURPOSE_MUTATE = 3, PURPOSE_LSPICK = 4, PURPOSE_LS = 5 };

typedef struct { uint32_t key[2]; uint32_t lig; } orc_rng;

static void rng_block(const orc_rng* r, int run, int ind, int gen, int purpose, int block, uint32_t w[4])
{
    uint32_t ctr[4] = {r->lig, ((uint32_t)run << 16) | (uint32_t)ind, (uint32_t)gen,
                       ((uint32_t)purpose << 20) | (uint32_t)block};
    orc_philox4x32_10(ctr, r->key, w);
}

/* u32 -> uniform in [0, 1): top 24 bits times 2^-24 (exact in float and double). */
static double u01(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }
/* u32 -> uniform in (0, 1] for the logarithm of Box-Muller. */
static double u01_open0(uint32_t x) { return (double)((x >> 8) + 1u) * (1.0 / 16777216.0); }
/* u32 -> index in [0, n) by multiply-shift. */
static int uindex(uint32_t x, int n) { return (int)(((uint64_t)x * (uint64_t)n) >> 32); }
/* probability test with an integer threshold floor(p * 2^24). */
static uint32_t prob_threshold(double p)
{
    if (p <= 0) return 0;
    if (p >= 1) return 16777216u;
    return (uint32_t)floor(p * 16777216.0);
}
static int ptest(uint32_t x, uint32_t thr) { return (x >> 8) < thr; }

/* ======================================================================== */
/* Pair potentials (AutoDock4 free-energy model, paper Sec. 1).             */
/* ======================================================================== */

/* Mehler-Solmajer distance-dependent dielectric:
 * eps(r) = A + B / (1 + k exp(-lambda B r)),  B = eps0 - A. */
static double ms_dielectric(const orc_ff* ff, double r)
{
    double B = ff->ms_eps0 - ff->ms_A;
    return ff->ms_A + B / (1.0 + ff->ms_k * exp(-ff->ms_lambda * B * r));
}

static double ms_dielectric_deriv(const orc_ff* ff, double r)
{
    double B = ff->ms_eps0 - ff->ms_A;
    double e = exp(-ff->ms_lambda * B * r);
    double den = 1.0 + ff->ms_k * e;
    return B * ff->ms_k * ff->ms_lambda * B * e / (den * den);
}

/* x^n for a small non-negative integer n, by repeated multiplication. */
static double ipow(double x, int n)
{
    double r = 1.0;
    for (int k = 0; k < n; ++k) r *= x;
    return r;
}

/* Is (ti, tj) a hydrogen-bond pair (donor HD with an acceptor)?  Returns the
 * acceptor's type or -1. */
static int hbond_acceptor(const orc_ff* ff, int ti, int tj)
{
    if (ff->hb_donor[ti] > 0.5 && ff->hb_acceptor[tj] > 0.5) return tj;
    if (ff->hb_donor[tj] > 0.5 && ff->hb_acceptor[ti] > 0.5) return ti;
    return -1;
}

/* Dispersion/repulsion or hydrogen bond, weighted, as a generalised n-m
 * potential with minimum -eps at r0:  C_n = m/(n-m) eps r0^n,
 * C_m = n/(n-m) eps r0^m.  12-6 for all pairs except donor-acceptor pairs,
 * which take 12-10 with the acceptor's r0 and eps.  r0 = (Ri + Rj)/2,
 * eps = sqrt(eps_i eps_j).  Value capped at +e_cap (reading), r floored at
 * r_min.  Returns energy; *dEdr receives dE/dr (0 where floored or capped). */
double orc_pair_lj(const orc_ff* ff, int ti, int tj, double r, double* dEdr)
{
    int acc = hbond_acceptor(ff, ti, tj);
    int n = 12, m;
    double eps, r0, w;
    if (acc >= 0) { m = 10; eps = ff->hb_eps[acc]; r0 = ff->hb_R[acc]; w = ff->w_hb; }
    else { m = 6; eps = sqrt(ff->epsii[ti] * ff->epsii[tj]); r0 = 0.5 * (ff->Rii[ti] + ff->Rii[tj]); w = ff->w_vdw; }
    double Cn = (double)m / (n - m) * eps * ipow(r0, n);
    double Cm = (double)n / (n - m) * eps * ipow(r0, m);
    int floored = r < ff->r_min;
    double rr = floored ? ff->r_min : r;
    double e = w * (Cn / ipow(rr, n) - Cm / ipow(rr, m));
    double d = w * (-n * Cn / ipow(rr, n + 1) + m * Cm / ipow(rr, m + 1));
    if (e > ff->e_cap) { e = ff->e_cap; d = 0.0; }
    if (floored) d = 0.0;
    if (dEdr) *dEdr = d;
    return e;
}

/* Coulomb with the Mehler-Solmajer dielectric, weighted:
 * w_elec * coulomb * qi qj / (eps(r) r), r floored at r_min. */
double orc_pair_elec(const orc_ff* ff, double qiqj, double r, double* dEdr)
{
    int floored = r < ff->r_min;
    double rr = floored ? ff->r_min : r;
    double eps = ms_dielectric(ff, rr);
    double c = ff->w_elec * ff->coulomb * qiqj;
    double e = c / (eps * rr);
    /* d/dr [1/(eps r)] = -(eps + r eps') / (eps r)^2 */
    double d = -c * (eps + rr * ms_dielectric_deriv(ff, rr)) / ((eps * rr) * (eps * rr));
    if (floored) d = 0.0;
    if (dEdr) *dEdr = d;
    return e;
}

/* AD4 desolvation pair term, weighted:
 * w_desolv [(S_i + qasp|q_i|) V_j + (S_j + qasp|q_j|) V_i] exp(-r^2 / (2 sigma^2)). */
double orc_pair_desolv(const orc_ff* ff, int ti, double qi, int tj, double qj, double r, double* dEdr)
{
    int floored = r < ff->r_min;
    double rr = floored ? ff->r_min : r;
    double coef = ff->w_desolv * ((ff->solpar[ti] + ff->qasp * fabs(qi)) * ff->vol[tj] +
                                  (ff->solpar[tj] + ff->qasp * fabs(qj)) * ff->vol[ti]);
    double s2 = ff->sigma * ff->sigma;
    double g = exp(-rr * rr / (2.0 * s2));
    double e = coef * g;
    double d = floored ? 0.0 : -coef * g * rr / s2;
    if (dEdr) *dEdr = d;
    return e;
}

/* ======================================================================== */
/* Grid maps (a0; AutoGrid4's role in the paper, Sec. 2.3).                  */
/* ======================================================================== */

/* Smooth receptor cutoff (reading): 1 below r_on, 0 above r_off,
 * 1 - 3u^2 + 2u^3 in between with u = (r - r_on)/(r_off - r_on). */
double orc_map_switch(const orc_ff* ff, double r)
{
    if (r <= ff->map_r_on) return 1.0;
    if (r >= ff->map_r_off) return 0.0;
    double u = (r - ff->map_r_on) / (ff->map_r_off - ff->map_r_on);
    return 1.0 - 3.0 * u * u + 2.0 * u * u * u;
}

/* Value of each map at one point p:
 *   M_t(p) = min(cap, sum_j S(r) [LJ/HB(t, type_j)(r) + w_d (S_t V_j + (S_j + qasp|q_j|) V_t) G(r)])
 *   M_e(p) = sum_j S(r) w_elec coulomb q_j / (eps(r) r)
 *   M_d(p) = sum_j S(r) w_desolv qasp V_j G(r)
 * A ligand atom of type t and charge q then scores M_t + q M_e + |q| M_d,
 * which reproduces the pair desolvation term above. */
void orc_map_point(const orc_ff* ff, const double p[3], int nrec, const double* rxyz,
                   const int* rtype, const double* rq, double out[ORC_NMAPS])
{
    double acc[ORC_NMAPS];
    for (int m = 0; m < ORC_NMAPS; ++m) acc[m] = 0.0;
    double s2 = ff->sigma * ff->sigma;
    for (int j = 0; j < nrec; ++j) {
        double dx = p[0] - rxyz[3 * j], dy = p[1] - rxyz[3 * j + 1], dz = p[2] - rxyz[3 * j + 2];
        double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 >= ff->map_r_off * ff->map_r_off) continue;   /* switch is exactly 0 there */
        double r = sqrt(r2);
        double sw = orc_map_switch(ff, r);
        if (sw == 0.0) continue;
        double rr = r < ff->r_min ? ff->r_min : r;
        double G = exp(-rr * rr / (2.0 * s2));
        int tj = rtype[j];
        for (int t = 0; t < ORC_NTYPES; ++t) {
            double e = orc_pair_lj(ff, t, tj, r, NULL);
            e += ff->w_desolv * (ff->solpar[t] * ff->vol[tj] + (ff->solpar[tj] + ff->qasp * fabs(rq[j])) * ff->vol[t]) * G;
            acc[t] += sw * e;
        }
        acc[ORC_MAP_ELEC] += sw * orc_pair_elec(ff, rq[j], r, NULL);
        acc[ORC_MAP_DESOLV] += sw * ff->w_desolv * ff->qasp * ff->vol[tj] * G;
    }
    for (int t = 0; t < ORC_NTYPES; ++t) if (acc[t] > ff->e_cap) acc[t] = ff->e_cap;
    for (int m = 0; m < ORC_NMAPS; ++m) out[m] = acc[m];
}

/* Full maps, layout [map][z][y][x], node (i,j,k) at origin + (i,j,k) h. */
void orc_maps_build(const orc_ff* ff, const orc_grid* g, int nrec, const double* rxyz,
                    const int* rtype, const double* rq, double* maps)
{
    size_t nx = g->n[0], ny = g->n[1], nz = g->n[2];
    size_t npt = nx * ny * nz;
    /* planes are independent; the loop is split over threads only */
    #pragma omp parallel for schedule(dynamic)
    for (size_t k = 0; k < nz; ++k)
        for (size_t j = 0; j < ny; ++j)
            for (size_t i = 0; i < nx; ++i) {
                double p[3] = {g->origin[0] + i * g->spacing, g->origin[1] + j * g->spacing,
                               g->origin[2] + k * g->spacing};
                double v[ORC_NMAPS];
                orc_map_point(ff, p, nrec, rxyz, rtype, rq, v);
                size_t idx = (k * ny + j) * nx + i;
                for (int m = 0; m < ORC_NMAPS; ++m) maps[m * npt + idx] = v[m];
            }
}

/* ======================================================================== */
/* Trilinear interpolation with the out-of-box penalty (reading).           */
/* ======================================================================== */

/* u = (p - o)/h per axis, with the point first clamped into the box;
 * i0 = floor(u) clamped to [0, n-2]; f = u - i0.  Value = sum over the 8
 * corners of the trilinear weights times the node values; gradient = the
 * derivative of the weights / h, zero along an axis where the point was
 * clamped (moving it there does not move the clamped point). */
double orc_trilinear(const orc_grid* g, const double* map, const double p[3], double grad[3])
{
    int nx = g->n[0], ny = g->n[1];
    int i0[3], clamped[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double lo = g->origin[a], hi = g->origin[a] + (g->n[a] - 1) * g->spacing;
        double pc = p[a];
        clamped[a] = 0;
        if (pc < lo) { pc = lo; clamped[a] = 1; }
        if (pc > hi) { pc = hi; clamped[a] = 1; }
        double u = (pc - g->origin[a]) / g->spacing;
        int i = (int)floor(u);
        if (i < 0) i = 0;
        if (i > g->n[a] - 2) i = g->n[a] - 2;
        i0[a] = i;
        f[a] = u - i;
    }
    double v = 0.0, dv[3] = {0, 0, 0};
    for (int c = 0; c < 8; ++c) {
        int bx = c & 1, by = (c >> 1) & 1, bz = (c >> 2) & 1;
        double wx = bx ? f[0] : 1.0 - f[0];
        double wy = by ? f[1] : 1.0 - f[1];
        double wz = bz ? f[2] : 1.0 - f[2];
        double sx = bx ? 1.0 : -1.0, sy = by ? 1.0 : -1.0, sz = bz ? 1.0 : -1.0;
        size_t idx = ((size_t)(i0[2] + bz) * ny + (i0[1] + by)) * nx + (i0[0] + bx);
        double m = map[idx];
        v += wx * wy * wz * m;
        dv[0] += sx * wy * wz * m;
        dv[1] += wx * sy * wz * m;
        dv[2] += wx * wy * sz * m;
    }
    for (int a = 0; a < 3; ++a) grad[a] = clamped[a] ? 0.0 : dv[a] / g->spacing;
    return v;
}

/* Out-of-box restraint (reading; the paper is silent): K d^2 with d the
 * distance from p to the box, and its gradient. */
double orc_out_of_box(const orc_grid* g, const double p[3], double k_out, double grad[3])
{
    double pen = 0.0;
    for (int a = 0; a < 3; ++a) {
        double lo = g->origin[a], hi = g->origin[a] + (g->n[a] - 1) * g->spacing;
        grad[a] = 0.0;
        if (p[a] < lo) { pen += (lo - p[a]) * (lo - p[a]); grad[a] = 2.0 * k_out * (p[a] - lo); }
        if (p[a] > hi) { pen += (p[a] - hi) * (p[a] - hi); grad[a] = 2.0 * k_out * (p[a] - hi); }
    }
    return k_out * pen;
}

/* ======================================================================== */
/* Ligand topology: rigid fragments, torsion subtrees, intramolecular pairs */
/* ======================================================================== */
typedef struct {
    int natoms, ntors, npairs;
    double xyz[ORC_MAXATOMS][3];
    int type[ORC_MAXATOMS];
    double q[ORC_MAXATOMS];
    double centroid[3];
    int tors_a[ORC_MAXTORS], tors_b[ORC_MAXTORS];   /* a on the root side      */
    unsigned char moving[ORC_MAXTORS][ORC_MAXATOMS]; /* S_k membership          */
    int depth[ORC_MAXTORS];                          /* ancestor torsion count  */
    int order[ORC_MAXTORS];                          /* deepest first           */
    int frag[ORC_MAXATOMS];
    int pair_i[ORC_MAXPAIRS], pair_j[ORC_MAXPAIRS];
} orc_ligand;

size_t orc_ligand_sizeof(void) { return sizeof(orc_ligand); }

/* Error codes shared with nothing: local to the oracle. */
#define ORC_OK 0
#define ORC_EINVAL -1

/* Build the topology.  Readings (the paper is silent on them):
 *  - a rotatable bond (a,b) moves the side of the tree not holding `root`;
 *  - rigid fragments = connected components once rotatable bonds are cut;
 *  - an intramolecular pair (i<j) is scored unless i and j are in the same
 *    rigid fragment or are at most 3 bonds apart (1-2, 1-3, 1-4). */
int orc_ligand_init(orc_ligand* L, int natoms, const double* xyz, const int* type, const double* q,
                    int nbonds, const int* bonds, int ntors, const int* tors, int root)
{
    if (natoms < 1 || natoms > ORC_MAXATOMS || ntors < 0 || ntors > ORC_MAXTORS || root < 0 || root >= natoms)
        return ORC_EINVAL;
    memset(L, 0, sizeof(*L));
    L->natoms = natoms;
    L->ntors = ntors;
    for (int i = 0; i < natoms; ++i) {
        for (int a = 0; a < 3; ++a) L->xyz[i][a] = xyz[3 * i + a];
        L->type[i] = type[i];
        L->q[i] = q[i];
        if (type[i] < 0 || type[i] >= ORC_NTYPES) return ORC_EINVAL;
    }
    for (int a = 0; a < 3; ++a) {
        double s = 0.0;
        for (int i = 0; i < natoms; ++i) s += xyz[3 * i + a];
        L->centroid[a] = s / natoms;
    }
    /* adjacency */
    int (*adj)[ORC_MAXATOMS] = calloc(ORC_MAXATOMS, sizeof(*adj));
    int (*dist)[ORC_MAXATOMS] = calloc(ORC_MAXATOMS, sizeof(*dist));
    int rc = ORC_OK, nf = 0, np = 0;
    int used[ORC_MAXTORS];
    for (int b = 0; b < nbonds; ++b) {
        int i = bonds[2 * b], j = bonds[2 * b + 1];
        if (i < 0 || j < 0 || i >= natoms || j >= natoms || i == j) { rc = ORC_EINVAL; goto done; }
        adj[i][j] = adj[j][i] = 1;
    }
    /* graph distances by repeated relaxation (Floyd-Warshall on unit edges) */
    for (int i = 0; i < natoms; ++i)
        for (int j = 0; j < natoms; ++j) dist[i][j] = (i == j) ? 0 : (adj[i][j] ? 1 : 100000);
    for (int k = 0; k < natoms; ++k)
        for (int i = 0; i < natoms; ++i)
            for (int j = 0; j < natoms; ++j)
                if (dist[i][k] + dist[k][j] < dist[i][j]) dist[i][j] = dist[i][k] + dist[k][j];
    for (int i = 0; i < natoms; ++i)
        if (dist[root][i] >= 100000) { rc = ORC_EINVAL; goto done; } /* not connected */
    /* torsions: moving side = atoms whose path from root passes through b
     * after a, i.e. reachable from b without using the bond (a,b). */
    for (int k = 0; k < ntors; ++k) {
        int a = tors[2 * k], b = tors[2 * k + 1];
        if (a < 0 || b < 0 || a >= natoms || b >= natoms || !adj[a][b]) { rc = ORC_EINVAL; goto done; }
        if (dist[root][b] < dist[root][a]) { int t = a; a = b; b = t; }
        L->tors_a[k] = a;
        L->tors_b[k] = b;
        /* flood fill from b, never crossing into a */
        int stack[ORC_MAXATOMS], sp = 0;
        L->moving[k][b] = 1;
        stack[sp++] = b;
        while (sp) {
            int u = stack[--sp];
            for (int v = 0; v < natoms; ++v)
                if (adj[u][v] && v != a && !L->moving[k][v]) { L->moving[k][v] = 1; stack[sp++] = v; }
        }
        if (L->moving[k][root]) { rc = ORC_EINVAL; goto done; } /* a cycle through the bond */
    }
    /* torsion depth = number of other torsions whose moving set contains b_k */
    for (int k = 0; k < ntors; ++k) {
        int d = 0;
        for (int j = 0; j < ntors; ++j)
            if (j != k && L->moving[j][L->tors_b[k]]) ++d;
        L->depth[k] = d;
    }
    /* deepest first (stable in torsion index) */
    memset(used, 0, sizeof(used));
    for (int s = 0; s < ntors; ++s) {
        int best = -1;
        for (int k = 0; k < ntors; ++k)
            if (!used[k] && (best < 0 || L->depth[k] > L->depth[best])) best = k;
        used[best] = 1;
        L->order[s] = best;
    }
    /* rigid fragments: components of the bond graph without rotatable bonds */
    for (int i = 0; i < natoms; ++i) L->frag[i] = -1;
    nf = 0;
    for (int s = 0; s < natoms; ++s) {
        if (L->frag[s] >= 0) continue;
        int stack[ORC_MAXATOMS], sp = 0;
        L->frag[s] = nf;
        stack[sp++] = s;
        while (sp) {
            int u = stack[--sp];
            for (int v = 0; v < natoms; ++v) {
                if (!adj[u][v] || L->frag[v] >= 0) continue;
                int rot = 0;
                for (int k = 0; k < ntors; ++k)
                    if ((L->tors_a[k] == u && L->tors_b[k] == v) || (L->tors_a[k] == v && L->tors_b[k] == u)) rot = 1;
                if (rot) continue;
                L->frag[v] = nf;
                stack[sp++] = v;
            }
        }
        ++nf;
    }
    /* intramolecular pair list */
    np = 0;
    for (int i = 0; i < natoms; ++i)
        for (int j = i + 1; j < natoms; ++j) {
            if (L->frag[i] == L->frag[j]) continue;
            if (dist[i][j] <= 3) continue;
            L->pair_i[np] = i;
            L->pair_j[np] = j;
            ++np;
        }
    L->npairs = np;
done:
    free(adj);
    free(dist);
    return rc;
}

int orc_ligand_npairs(const orc_ligand* L) { return L->npairs; }
void orc_ligand_pairs(const orc_ligand* L, int* ij)
{
    for (int p = 0; p < L->npairs; ++p) { ij[2 * p] = L->pair_i[p]; ij[2 * p + 1] = L->pair_j[p]; }
}
void orc_ligand_moving(const orc_ligand* L, unsigned char* mv)
{
    for (int k = 0; k < L->ntors; ++k)
        for (int i = 0; i < L->natoms; ++i) mv[k * L->natoms + i] = L->moving[k][i];
}
void orc_ligand_torsions(const orc_ligand* L, int* ab)
{
    for (int k = 0; k < L->ntors; ++k) { ab[2 * k] = L->tors_a[k]; ab[2 * k + 1] = L->tors_b[k]; }
}

/* ======================================================================== */
/* Genotype -> pose (paper Sec. 1: LGA genotype; pose details are readings). */
/* Genes: t[3] (A), q[4] = (w, x, y, z) used as q/|q|, theta[T] (rad) as     */
/* deltas from the input conformation.                                        */
/* ======================================================================== */

/* Rotation matrix of a unit quaternion (w, x, y, z): x' = q (0,x) q*. */
void orc_quat_to_matrix(const double qin[4], double R[3][3])
{
    double n = sqrt(qin[0] * qin[0] + qin[1] * qin[1] + qin[2] * qin[2] + qin[3] * qin[3]);
    double w = qin[0] / n, x = qin[1] / n, y = qin[2] / n, z = qin[3] / n;
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

/* Rotate point p about the axis through `a` with unit direction u by angle
 * th (right-hand rule), Rodrigues' formula. */
static void rotate_about(const double a[3], const double u[3], double th, double p[3])
{
    double v[3] = {p[0] - a[0], p[1] - a[1], p[2] - a[2]};
    double c = cos(th), s = sin(th);
    double uxv[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
    double udv = u[0] * v[0] + u[1] * v[1] + u[2] * v[2];
    for (int k = 0; k < 3; ++k) p[k] = a[k] + v[k] * c + uxv[k] * s + u[k] * udv * (1 - c);
}

/* Pose: apply the torsions deepest first in the ligand frame, each rotating
 * its moving set S_k about the reference axis a_k -> b_k by theta_k; then
 * x' = R(q/|q|)(x - c) + t with c the reference centroid. */
void orc_pose(const orc_ligand* L, const double* genes, double* out_xyz)
{
    double x[ORC_MAXATOMS][3];
    for (int i = 0; i < L->natoms; ++i)
        for (int a = 0; a < 3; ++a) x[i][a] = L->xyz[i][a];
    for (int s = 0; s < L->ntors; ++s) {
        int k = L->order[s];
        const double* pa = L->xyz[L->tors_a[k]];
        const double* pb = L->xyz[L->tors_b[k]];
        double u[3] = {pb[0] - pa[0], pb[1] - pa[1], pb[2] - pa[2]};
        double n = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        for (int a = 0; a < 3; ++a) u[a] /= n;
        for (int i = 0; i < L->natoms; ++i)
            if (L->moving[k][i]) rotate_about(pa, u, genes[7 + k], x[i]);
    }
    double R[3][3];
    orc_quat_to_matrix(genes + 3, R);
    for (int i = 0; i < L->natoms; ++i) {
        double d[3] = {x[i][0] - L->centroid[0], x[i][1] - L->centroid[1], x[i][2] - L->centroid[2]};
        for (int a = 0; a < 3; ++a)
            out_xyz[3 * i + a] = R[a][0] * d[0] + R[a][1] * d[1] + R[a][2] * d[2] + genes[a];
    }
}

/* ======================================================================== */
/* Energy and gradient of one genotype.                                      */
/* ======================================================================== */
typedef struct {
    double e_total, e_inter, e_intra;
    double grad_genes[ORC_MAXGENES];   /* dE/dt, dE/dq (4), dE/dtheta */
    double grad_tangent[ORC_MAXGENES]; /* dE/dt, torque dE/domega (3), dE/dtheta */
} orc_score_out;

/* Intermolecular part for atom i at x: M_t + q M_e + |q| M_d + K d^2. */
static double atom_inter(const orc_ff* ff, const orc_grid* g, const double* maps, int t, double q,
                         const double x[3], double grad[3])
{
    size_t npt = (size_t)g->n[0] * g->n[1] * g->n[2];
    double gt[3], ge[3], gd[3], gp[3];
    double vt = orc_trilinear(g, maps + (size_t)t * npt, x, gt);
    double ve = orc_trilinear(g, maps + (size_t)ORC_MAP_ELEC * npt, x, ge);
    double vd = orc_trilinear(g, maps + (size_t)ORC_MAP_DESOLV * npt, x, gd);
    double pen = orc_out_of_box(g, x, ff->k_out, gp);
    for (int a = 0; a < 3; ++a) grad[a] = gt[a] + q * ge[a] + fabs(q) * gd[a] + gp[a];
    return vt + q * ve + fabs(q) * vd + pen;
}

/* Energy of posed coordinates x (natoms x 3): E_inter + E_intra (the search
 * objective; reading) and the per-atom gradient f_i = dE/dx_i.  The
 * intermolecular part sums, per atom, the trilinear maps plus the out-of-box
 * restraint; the intramolecular part sums the three pair terms over the
 * pair list, each pair's dE/dr applied along the unit vector between the
 * two atoms (Sec. 1: vdW / H-bond, electrostatic and desolvation terms). */
static void score_coords(const orc_ff* ff, const orc_grid* g, const double* maps, const orc_ligand* L,
                         const double* x, double* e_inter_out, double* e_intra_out, double (*f)[3])
{
    int n = L->natoms;
    double e_inter = 0.0, e_intra = 0.0;
    for (int i = 0; i < n; ++i) {
        double gi[3];
        e_inter += atom_inter(ff, g, maps, L->type[i], L->q[i], x + 3 * i, gi);
        for (int a = 0; a < 3; ++a) f[i][a] = gi[a];
    }
    for (int p = 0; p < L->npairs; ++p) {
        int i = L->pair_i[p], j = L->pair_j[p];
        double d[3] = {x[3 * i] - x[3 * j], x[3 * i + 1] - x[3 * j + 1], x[3 * i + 2] - x[3 * j + 2]};
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double d1, d2, d3;
        double e = orc_pair_lj(ff, L->type[i], L->type[j], r, &d1) +
                   orc_pair_elec(ff, L->q[i] * L->q[j], r, &d2) +
                   orc_pair_desolv(ff, L->type[i], L->q[i], L->type[j], L->q[j], r, &d3);
        e_intra += e;
        double dEdr = d1 + d2 + d3;
        if (r > 0.0) {
            for (int a = 0; a < 3; ++a) {
                f[i][a] += dEdr * d[a] / r;
                f[j][a] -= dEdr * d[a] / r;
            }
        }
    }
    *e_inter_out = e_inter;
    *e_intra_out = e_intra;
}

/* Total energy of a genotype and its gradient: pose (orc_pose), then the
 * energy of the posed coordinates (score_coords) with g_i = dE/dx'_i, then
 *   dE/dt = sum_i g_i
 *   torque = sum_i (x'_i - t) x g_i                (tangent of a world-frame rotation)
 *   dE/dtheta_k = sum_{i in S_k} (u'_k x (x'_i - x'_{a_k})) . g_i, u'_k the posed axis
 *   dE/dq = 2 (-tau.v, w tau + tau x v) / |q|, with q/|q| = (w, v)   (chain rule
 *           through x' = q (0,x) q*: the derivative of a unit-quaternion rotation
 *           with respect to q is a rotation generator, projected off the
 *           radial direction by the normalisation). */
int orc_score(const orc_ff* ff, const orc_grid* g, const double* maps, const orc_ligand* L,
              const double* genes, orc_score_out* out, double* xyz_out)
{
    int n = L->natoms;
    double x[ORC_MAXATOMS * 3];
    double f[ORC_MAXATOMS][3];
    orc_pose(L, genes, x);
    double e_inter, e_intra;
    score_coords(ff, g, maps, L, x, &e_inter, &e_intra, f);
    double gt[3] = {0, 0, 0}, tau[3] = {0, 0, 0};
    for (int i = 0; i < n; ++i) {
        double rel[3] = {x[3 * i] - genes[0], x[3 * i + 1] - genes[1], x[3 * i + 2] - genes[2]};
        for (int a = 0; a < 3; ++a) gt[a] += f[i][a];
        tau[0] += rel[1] * f[i][2] - rel[2] * f[i][1];
        tau[1] += rel[2] * f[i][0] - rel[0] * f[i][2];
        tau[2] += rel[0] * f[i][1] - rel[1] * f[i][0];
    }
    double gth[ORC_MAXTORS];
    for (int k = 0; k < L->ntors; ++k) {
        const double* xa = x + 3 * L->tors_a[k];
        const double* xb = x + 3 * L->tors_b[k];
        double u[3] = {xb[0] - xa[0], xb[1] - xa[1], xb[2] - xa[2]};
        double un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        for (int a = 0; a < 3; ++a) u[a] /= un;
        double s = 0.0;
        for (int i = 0; i < n; ++i) {
            if (!L->moving[k][i]) continue;
            double v[3] = {x[3 * i] - xa[0], x[3 * i + 1] - xa[1], x[3 * i + 2] - xa[2]};
            double c[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
            s += c[0] * f[i][0] + c[1] * f[i][1] + c[2] * f[i][2];
        }
        gth[k] = s;
    }
    double qn = sqrt(genes[3] * genes[3] + genes[4] * genes[4] + genes[5] * genes[5] + genes[6] * genes[6]);
    double w = genes[3] / qn, v[3] = {genes[4] / qn, genes[5] / qn, genes[6] / qn};
    double tdv = tau[0] * v[0] + tau[1] * v[1] + tau[2] * v[2];
    double txv[3] = {tau[1] * v[2] - tau[2] * v[1], tau[2] * v[0] - tau[0] * v[2], tau[0] * v[1] - tau[1] * v[0]};
    out->e_inter = e_inter;
    out->e_intra = e_intra;
    out->e_total = e_inter + e_intra;
    for (int a = 0; a < 3; ++a) { out->grad_genes[a] = gt[a]; out->grad_tangent[a] = gt[a]; }
    out->grad_genes[3] = -2.0 * tdv / qn;
    for (int a = 0; a < 3; ++a) out->grad_genes[4 + a] = 2.0 * (w * tau[a] + txv[a]) / qn;
    for (int a = 0; a < 3; ++a) out->grad_tangent[3 + a] = tau[a];
    for (int k = 0; k < L->ntors; ++k) { out->grad_genes[7 + k] = gth[k]; out->grad_tangent[6 + k] = gth[k]; }
    if (xyz_out) memcpy(xyz_out, x, sizeof(double) * 3 * n);
    return ORC_OK;
}

/* Per-atom gradients dE/dx'_i of npose genotypes -> forces[npose][natoms][3]
 * (used by the tests to bound how FP32 rounding of the coordinates moves
 * the energy). */
void orc_atom_gradients(const orc_ff* ff, const orc_grid* g, const double* maps, const orc_ligand* L,
                        const double* genes, int npose, double* forces)
{
    int n = L->natoms, G = 7 + L->ntors;
    for (int p = 0; p < npose; ++p) {
        double x[ORC_MAXATOMS * 3], f[ORC_MAXATOMS][3], ei, ea;
        orc_pose(L, genes + (size_t)p * G, x);
        score_coords(ff, g, maps, L, x, &ei, &ea, f);
        memcpy(forces + (size_t)p * n * 3, f, sizeof(double) * 3 * n);
    }
}

/* Energies of npose sets of posed coordinates xyz[npose][natoms][3], given
 * directly rather than as genotypes (the same sums as orc_score after its
 * pose step): total and intermolecular energy per pose, and optionally the
 * per-atom gradients forces[npose][natoms][3].  Lets the tests separate the
 * rounding of the posed coordinates from the rounding of the scoring sums. */
void orc_score_xyz(const orc_ff* ff, const orc_grid* g, const double* maps, const orc_ligand* L,
                   const double* xyz, int npose, double* energy, double* e_inter, double* forces)
{
    int n = L->natoms;
    for (int p = 0; p < npose; ++p) {
        double f[ORC_MAXATOMS][3], ei, ea;
        score_coords(ff, g, maps, L, xyz + (size_t)p * n * 3, &ei, &ea, f);
        if (energy) energy[p] = ei + ea;
        if (e_inter) e_inter[p] = ei;
        if (forces) memcpy(forces + (size_t)p * n * 3, f, sizeof(double) * 3 * n);
    }
}

/* Batch form for the tests: npose genotypes (stride 7+T) -> energies and
 * gene gradients (stride 7+T) and tangent gradients (stride 6+T). */
void orc_score_batch(const orc_ff* ff, const orc_grid* g, const double* maps, const orc_ligand* L,
                     const double* genes, int npose, double* energy, double* e_inter, double* grad_genes,
                     double* grad_tangent)
{
    int G = 7 + L->ntors, D = 6 + L->ntors;
    for (int p = 0; p < npose; ++p) {
        orc_score_out o;
        orc_score(ff, g, maps, L, genes + (size_t)p * G, &o, NULL);
        if (energy) energy[p] = o.e_total;
        if (e_inter) e_inter[p] = o.e_inter;
        if (grad_genes) memcpy(grad_genes + (size_t)p * G, o.grad_genes, sizeof(double) * G);
        if (grad_tangent) memcpy(grad_tangent + (size_t)p * D, o.grad_tangent, sizeof(double) * D);
    }
}

void orc_pose_batch(const orc_ligand* L, const double* genes, int npose, double* xyz)
{
    int G = 7 + L->ntors;
    for (int p = 0; p < npose; ++p) orc_pose(L, genes + (size_t)p * G, xyz + (size_t)p * 3 * L->natoms);
}

/* ======================================================================== */
/* Moves in the tangent space (reading): x (+) xi means t += xi_t,          */
/* q <- exp(xi_omega) (x) q (world-frame rotation vector, then q normalised),*/
/* theta += xi_theta.                                                        */
/* ======================================================================== */
static void quat_mul(const double a[4], const double b[4], double out[4])
{
    double r[4];
    r[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    r[1] = a[0] * b[1] + b[0] * a[1] + a[2] * b[3] - a[3] * b[2];
    r[2] = a[0] * b[2] + b[0] * a[2] + a[3] * b[1] - a[1] * b[3];
    r[3] = a[0] * b[3] + b[0] * a[3] + a[1] * b[2] - a[2] * b[1];
    memcpy(out, r, sizeof(r));
}

static void quat_from_rotvec(const double w[3], double q[4])
{
    double ang = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    if (ang < 1e-12) { q[0] = 1.0; q[1] = 0.5 * w[0]; q[2] = 0.5 * w[1]; q[3] = 0.5 * w[2]; return; }
    double s = sin(0.5 * ang) / ang;
    q[0] = cos(0.5 * ang); q[1] = s * w[0]; q[2] = s * w[1]; q[3] = s * w[2];
}

static void quat_normalise(double q[4])
{
    double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int a = 0; a < 4; ++a) q[a] /= n;
}

void orc_apply_step(int ntors, const double* genes, const double* xi, double sign, double* out)
{
    int G = 7 + ntors;
    memcpy(out, genes, sizeof(double) * G);
    for (int a = 0; a < 3; ++a) out[a] = genes[a] + sign * xi[a];
    double w[3] = {sign * xi[3], sign * xi[4], sign * xi[5]}, dq[4];
    quat_from_rotvec(w, dq);
    quat_mul(dq, genes + 3, out + 3);
    quat_normalise(out + 3);
    for (int k = 0; k < ntors; ++k) out[7 + k] = genes[7 + k] + sign * xi[6 + k];
}

/* ======================================================================== */
/* Search parameters and local search.                                      */
/* ======================================================================== */
typedef struct {
    int nrun, pop_size, nev, max_gen, ls_method; /* ls_method: 0 none, 1 Solis-Wets, 2 ADADELTA */
    int ls_max_iters, elitism;
    double ls_rate, crossover_rate, mutation_rate, tournament_rate;
    double sw_rho0, sw_rho_min, sw_expand, sw_contract;
    int sw_succ, sw_fail;
    double sw_scale_t, sw_scale_rot, sw_scale_tors;
    double ad_rho, ad_eps;
    double mut_t, mut_rot, mut_tors;   /* half-widths of the mutation draws */
    uint32_t seed_lo, seed_hi, lig_id;
    int autostop;                      /* stop a run early (paper Sec. 1.1) */
    double stopstd;                    /* ... when the std-dev of its best energy over 10 generations is below this */
} orc_params;

typedef struct {
    const orc_ff* ff;
    const orc_grid* g;
    const double* maps;
    const orc_ligand* L;
    long long evals;
} orc_problem;

static double eval_energy(orc_problem* P, const double* genes)
{
    orc_score_out o;
    orc_score(P->ff, P->g, P->maps, P->L, genes, &o, NULL);
    P->evals += 1;
    return o.e_total;
}

/* Box-Muller Gaussian for tangent dimension d in iteration `iter` of the
 * Solis-Wets search of (run, ind) in generation gen.  Block iter*8 + d/4;
 * the pair (d/2)%2 of the block's words gives (z_cos, z_sin). */
static double ls_gauss(const orc_rng* r, int run, int ind, int gen, int iter, int d)
{
    uint32_t w[4];
    rng_block(r, run, ind, gen, PURPOSE_LS, iter * 8 + d / 4, w);
    int p = (d / 2) % 2;
    double u1 = u01_open0(w[2 * p]), u2 = u01(w[2 * p + 1]);
    double rad = sqrt(-2.0 * log(u1));
    return (d % 2 == 0) ? rad * cos(2.0 * ORC_PI * u2) : rad * sin(2.0 * ORC_PI * u2);
}

/* Solis & Wets (1981) adaptive random search: trial xi = bias + rho s (.) z.
 * Accept x (+) xi if better (bias <- 0.4 xi + 0.2 bias), else try x (-) xi
 * (bias <- bias - 0.4 xi), else bias <- 0.5 bias.  rho doubles after
 * sw_succ consecutive successes and halves after sw_fail consecutive
 * failures; stop when rho < rho_min or after max_iters iterations.
 * trace (optional, for the tests): per iteration ORC_SW_TRACE_WIDTH doubles
 * = rho of the iteration, outcome (+1 x (+) xi accepted, -1 x (-) xi
 * accepted, 0 rejected), energy after it, xi[ORC_MAXGENES],
 * bias after it[ORC_MAXGENES]. */
#define ORC_SW_TRACE_WIDTH (3 + 2 * ORC_MAXGENES)
static int solis_wets(orc_problem* P, const orc_params* prm, const orc_rng* r, int run, int ind, int gen,
                      double* genes, double* energy, double* trace)
{
    int T = P->L->ntors, D = 6 + T, G = 7 + T;
    double bias[ORC_MAXGENES] = {0}, xi[ORC_MAXGENES], cand[ORC_MAXGENES];
    double rho = prm->sw_rho0;
    int succ = 0, fail = 0, it;
    double e = *energy;
    for (it = 0; it < prm->ls_max_iters && rho >= prm->sw_rho_min; ++it) {
        double rho_it = rho;
        int outcome;
        for (int d = 0; d < D; ++d) {
            double s = d < 3 ? prm->sw_scale_t : (d < 6 ? prm->sw_scale_rot : prm->sw_scale_tors);
            xi[d] = bias[d] + rho * s * ls_gauss(r, run, ind, gen, it, d);
        }
        orc_apply_step(T, genes, xi, +1.0, cand);
        double e1 = eval_energy(P, cand);
        if (e1 < e) {
            memcpy(genes, cand, sizeof(double) * G);
            e = e1;
            for (int d = 0; d < D; ++d) bias[d] = 0.4 * xi[d] + 0.2 * bias[d];
            ++succ; fail = 0;
            outcome = 1;
        } else {
            orc_apply_step(T, genes, xi, -1.0, cand);
            double e2 = eval_energy(P, cand);
            if (e2 < e) {
                memcpy(genes, cand, sizeof(double) * G);
                e = e2;
                for (int d = 0; d < D; ++d) bias[d] = bias[d] - 0.4 * xi[d];
                ++succ; fail = 0;
                outcome = -1;
            } else {
                for (int d = 0; d < D; ++d) bias[d] *= 0.5;
                ++fail; succ = 0;
                outcome = 0;
            }
        }
        if (succ >= prm->sw_succ) { rho *= prm->sw_expand; succ = 0; }
        if (fail >= prm->sw_fail) { rho *= prm->sw_contract; fail = 0; }
        if (trace) {
            double* t = trace + (size_t)it * ORC_SW_TRACE_WIDTH;
            memset(t, 0, sizeof(double) * ORC_SW_TRACE_WIDTH);
            t[0] = rho_it;
            t[1] = outcome;
            t[2] = e;
            for (int d = 0; d < D; ++d) { t[3 + d] = xi[d]; t[3 + ORC_MAXGENES + d] = bias[d]; }
        }
    }
    *energy = e;
    return it;
}

/* ADADELTA (Zeiler 2012) in the tangent space: per iteration evaluate E and
 * g at x, keep the best genotype seen, then
 *   Eg2 <- rho Eg2 + (1-rho) g^2
 *   dx  = -sqrt(Edx2 + eps) / sqrt(Eg2 + eps) * g
 *   Edx2 <- rho Edx2 + (1-rho) dx^2
 *   x <- x (+) dx.
 * One energy+gradient call = one evaluation. */
static void adadelta(orc_problem* P, const orc_params* prm, double* genes, double* energy)
{
    int T = P->L->ntors, D = 6 + T, G = 7 + T;
    double Eg2[ORC_MAXGENES] = {0}, Edx2[ORC_MAXGENES] = {0}, dx[ORC_MAXGENES];
    double x[ORC_MAXGENES], best[ORC_MAXGENES], nx[ORC_MAXGENES];
    memcpy(x, genes, sizeof(double) * G);
    memcpy(best, genes, sizeof(double) * G);
    double ebest = *energy;
    for (int it = 0; it < prm->ls_max_iters; ++it) {
        orc_score_out o;
        orc_score(P->ff, P->g, P->maps, P->L, x, &o, NULL);
        P->evals += 1;
        if (o.e_total < ebest) { ebest = o.e_total; memcpy(best, x, sizeof(double) * G); }
        for (int d = 0; d < D; ++d) {
            double gd = o.grad_tangent[d];
            Eg2[d] = prm->ad_rho * Eg2[d] + (1.0 - prm->ad_rho) * gd * gd;
            dx[d] = -sqrt(Edx2[d] + prm->ad_eps) / sqrt(Eg2[d] + prm->ad_eps) * gd;
            Edx2[d] = prm->ad_rho * Edx2[d] + (1.0 - prm->ad_rho) * dx[d] * dx[d];
        }
        orc_apply_step(T, x, dx, +1.0, nx);
        memcpy(x, nx, sizeof(double) * G);
    }
    memcpy(genes, best, sizeof(double) * G);
    *energy = ebest;
}

/* Local search on one genotype, exported for the tests. */
long long orc_local_search(const orc_ff* ff, const orc_grid* g, const double* maps, const orc_ligand* L,
                           const orc_params* prm, int run, int ind, int gen, double* genes, double* energy)
{
    orc_problem P = {ff, g, maps, L, 0};
    orc_rng r = {{prm->seed_lo, prm->seed_hi}, prm->lig_id};
    if (prm->ls_method == 1) solis_wets(&P, prm, &r, run, ind, gen, genes, energy, NULL);
    else if (prm->ls_method == 2) adadelta(&P, prm, genes, energy);
    return P.evals;
}

/* Solis-Wets on one genotype with its per-iteration trace (see solis_wets);
 * returns the number of iterations, *nevals the energy evaluations. */
int orc_solis_wets_trace(const orc_ff* ff, const orc_grid* g, const double* maps, const orc_ligand* L,
                         const orc_params* prm, int run, int ind, int gen, double* genes, double* energy,
                         double* trace, long long* nevals)
{
    orc_problem P = {ff, g, maps, L, 0};
    orc_rng r = {{prm->seed_lo, prm->seed_hi}, prm->lig_id};
    int iters = solis_wets(&P, prm, &r, run, ind, gen, genes, energy, trace);
    *nevals = P.evals;
    return iters;
}

/* ======================================================================== */
/* Lamarckian GA (paper Sec. 1): one run.                                   */
/* ======================================================================== */

/* Random initial genotype: t uniform in the grid box, q uniform on S^3
 * (Shoemake 1992, three uniforms), theta uniform in [-pi, pi). */
static void init_individual(const orc_rng* r, const orc_grid* g, int T, int run, int ind, double* genes)
{
    uint32_t w[4];
    rng_block(r, run, ind, 0, PURPOSE_INIT, 0, w);
    for (int a = 0; a < 3; ++a)
        genes[a] = g->origin[a] + u01(w[a]) * ((g->n[a] - 1) * g->spacing);
    rng_block(r, run, ind, 0, PURPOSE_INIT, 1, w);
    double u1 = u01(w[0]), u2 = u01(w[1]), u3 = u01(w[2]);
    double s1 = sqrt(1.0 - u1), s2 = sqrt(u1);
    genes[3] = s2 * cos(2.0 * ORC_PI * u3);
    genes[4] = s1 * sin(2.0 * ORC_PI * u2);
    genes[5] = s1 * cos(2.0 * ORC_PI * u2);
    genes[6] = s2 * sin(2.0 * ORC_PI * u3);
    for (int k = 0; k < T; ++k) {
        rng_block(r, run, ind, 0, PURPOSE_INIT, 2 + k / 4, w);
        genes[7 + k] = -ORC_PI + 2.0 * ORC_PI * u01(w[k % 4]);
    }
}

/* Per-offspring trace of the GA decisions, for the bit-exact replay test. */
typedef struct {
    int32_t parent1, parent2, xlo, xhi; /* xlo = xhi = -1 when no crossover */
    int32_t mut_mask, ls_applied;
    int32_t cand[4];                    /* tournament candidates a1, b1, a2, b2 (-1 for the elite) */
    int32_t pad0, pad1;
} orc_trace;

/* Binary tournament: two uniform indices; the better (lower energy, ties to
 * the lower index) wins with probability tournament_rate. */
static int tournament(const double* E, int pop, uint32_t wa, uint32_t wb, uint32_t wwin, uint32_t thr, int32_t* cand)
{
    int a = uindex(wa, pop), b = uindex(wb, pop);
    cand[0] = a;
    cand[1] = b;
    int better, worse;
    if (E[a] < E[b] || (E[a] == E[b] && a <= b)) { better = a; worse = b; }
    else { better = b; worse = a; }
    return ptest(wwin, thr) ? better : worse;
}

/* Build offspring `ind` of generation `gen` from population (Pg, Pe).
 * Gene blocks: [t], [q], [theta_1] ... [theta_T].  Two-point crossover over
 * blocks with probability crossover_rate: blocks in [lo, hi) come from the
 * second parent.  Each block mutates with probability mutation_rate:
 * t += U(-mut_t, mut_t) per component; q <- q_rot(axis, U(-mut_rot, mut_rot)) q
 * with a uniform random axis; theta += U(-mut_tors, mut_tors). */
static void make_offspring(const orc_rng* r, const orc_params* prm, int T, int run, int ind, int gen,
                           const double* Pg, const double* Pe, double* child, orc_trace* tr)
{
    int G = 7 + T, nb = 2 + T;
    uint32_t w[4];
    uint32_t thr_t = prob_threshold(prm->tournament_rate);
    int32_t cand[4];
    rng_block(r, run, ind, gen, PURPOSE_SELECT, 0, w);
    int p1 = tournament(Pe, prm->pop_size, w[0], w[1], w[2], thr_t, cand);
    rng_block(r, run, ind, gen, PURPOSE_SELECT, 1, w);
    int p2 = tournament(Pe, prm->pop_size, w[0], w[1], w[2], thr_t, cand + 2);
    rng_block(r, run, ind, gen, PURPOSE_SELECT, 2, w);
    int lo = -1, hi = -1;
    memcpy(child, Pg + (size_t)p1 * G, sizeof(double) * G);
    if (ptest(w[0], prob_threshold(prm->crossover_rate))) {
        int c1 = uindex(w[1], nb + 1), c2 = uindex(w[2], nb + 1);
        lo = c1 < c2 ? c1 : c2;
        hi = c1 < c2 ? c2 : c1;
        for (int b = lo; b < hi; ++b) {
            if (b == 0) for (int a = 0; a < 3; ++a) child[a] = Pg[(size_t)p2 * G + a];
            else if (b == 1) for (int a = 0; a < 4; ++a) child[3 + a] = Pg[(size_t)p2 * G + 3 + a];
            else child[7 + (b - 2)] = Pg[(size_t)p2 * G + 7 + (b - 2)];
        }
    }
    int mask = 0;
    uint32_t thr_m = prob_threshold(prm->mutation_rate);
    for (int b = 0; b < nb; ++b) {
        rng_block(r, run, ind, gen, PURPOSE_SELECT, 3 + b / 4, w);
        if (!ptest(w[b % 4], thr_m)) continue;
        mask |= 1 << b;
        uint32_t m[4];
        rng_block(r, run, ind, gen, PURPOSE_MUTATE, b, m);
        if (b == 0) {
            for (int a = 0; a < 3; ++a) child[a] += prm->mut_t * (2.0 * u01(m[a]) - 1.0);
        } else if (b == 1) {
            double z = 2.0 * u01(m[0]) - 1.0, phi = 2.0 * ORC_PI * u01(m[1]);
            double s = sqrt(1.0 - z * z);
            double ang = prm->mut_rot * (2.0 * u01(m[2]) - 1.0);
            double rv[3] = {ang * s * cos(phi), ang * s * sin(phi), ang * z}, dq[4], nq[4];
            quat_from_rotvec(rv, dq);
            quat_mul(dq, child + 3, nq);
            quat_normalise(nq);
            memcpy(child + 3, nq, sizeof(nq));
        } else {
            child[7 + (b - 2)] += prm->mut_tors * (2.0 * u01(m[0]) - 1.0);
        }
    }
    if (tr) {
        tr->parent1 = p1; tr->parent2 = p2; tr->xlo = lo; tr->xhi = hi; tr->mut_mask = mask;
        for (int k = 0; k < 4; ++k) tr->cand[k] = cand[k];
    }
}

/* make_offspring exported for the tests: offspring `ind` of generation `gen`
 * from the population genes Pg[pop][7+T] and energies Pe[pop]; the decision
 * record goes to *tr. */
void orc_make_offspring(const orc_params* prm, int T, int run, int ind, int gen, const double* Pg,
                        const double* Pe, double* child, orc_trace* tr)
{
    orc_rng r = {{prm->seed_lo, prm->seed_hi}, prm->lig_id};
    orc_trace t = {-1, -1, -1, -1, 0, 0, {-1, -1, -1, -1}, 0, 0};
    make_offspring(&r, prm, T, run, ind, gen, Pg, Pe, child, &t);
    *tr = t;
}

typedef struct {
    double best_energy;
    double best_genes[ORC_MAXGENES];
    long long evals;
    int generations;
    int pad;
} orc_run_result;

/* One LGA run.  Population init + evaluation, then generations while
 * evals < nev (the last one may overshoot) and gen < max_gen:
 *   elitism: offspring 0 = best of the previous population (copied, not
 *   re-evaluated); offspring 1.. from selection, crossover, mutation, each
 *   evaluated; then local search on each individual with probability
 *   ls_rate, the refined genotype written back (Lamarckian).
 * Optional outputs: trace[gen-1][ind] for the first ntrace generations and
 * the population after each traced generation (genes, energies). */
int orc_lga_run(const orc_ff* ff, const orc_grid* g, const double* maps, const orc_ligand* L,
                const orc_params* prm, int run, orc_run_result* res, int ntrace, orc_trace* trace,
                double* trace_genes, double* trace_energy)
{
    int T = L->ntors, G = 7 + T, pop = prm->pop_size;
    if (pop < 2 || pop > 65535 || T > ORC_MAXTORS) return ORC_EINVAL;
    orc_problem P = {ff, g, maps, L, 0};
    orc_rng r = {{prm->seed_lo, prm->seed_hi}, prm->lig_id};
    double* Pg = (double*)malloc(sizeof(double) * G * pop);
    double* Pe = (double*)malloc(sizeof(double) * pop);
    double* Ng = (double*)malloc(sizeof(double) * G * pop);
    double* Ne = (double*)malloc(sizeof(double) * pop);
    for (int i = 0; i < pop; ++i) {
        init_individual(&r, g, T, run, i, Pg + (size_t)i * G);
        Pe[i] = eval_energy(&P, Pg + (size_t)i * G);
    }
    int gen = 0;
    uint32_t thr_ls = prob_threshold(prm->ls_rate);
    double hist[10];                   /* best energy after each of the last 10 generations */
    while (P.evals < prm->nev && gen < prm->max_gen) {
        ++gen;
        int elite = 0;
        for (int i = 1; i < pop; ++i) if (Pe[i] < Pe[elite]) elite = i;
        for (int i = 0; i < pop; ++i) {
            orc_trace tr = {-1, -1, -1, -1, 0, 0, {-1, -1, -1, -1}, 0, 0};
            double* child = Ng + (size_t)i * G;
            if (i < prm->elitism) {
                memcpy(child, Pg + (size_t)elite * G, sizeof(double) * G);
                Ne[i] = Pe[elite];
                tr.parent1 = tr.parent2 = elite;
            } else {
                make_offspring(&r, prm, T, run, i, gen, Pg, Pe, child, &tr);
                Ne[i] = eval_energy(&P, child);
            }
            uint32_t w[4];
            rng_block(&r, run, i, gen, PURPOSE_LSPICK, 0, w);
            if (prm->ls_method != 0 && ptest(w[0], thr_ls)) {
                tr.ls_applied = 1;
                if (prm->ls_method == 1) solis_wets(&P, prm, &r, run, i, gen, child, &Ne[i], NULL);
                else adadelta(&P, prm, child, &Ne[i]);
            }
            if (trace && gen <= ntrace) trace[(size_t)(gen - 1) * pop + i] = tr;
        }
        memcpy(Pg, Ng, sizeof(double) * G * pop);
        memcpy(Pe, Ne, sizeof(double) * pop);
        if (gen <= ntrace) {
            if (trace_genes) memcpy(trace_genes + (size_t)(gen - 1) * pop * G, Pg, sizeof(double) * G * pop);
            if (trace_energy) memcpy(trace_energy + (size_t)(gen - 1) * pop, Pe, sizeof(double) * pop);
        }
        /* autostop (paper Sec. 1.1; reading: population standard deviation of
         * the best energy over the last 10 generations, compared to stopstd) */
        double b = Pe[0];
        for (int i = 1; i < pop; ++i) if (Pe[i] < b) b = Pe[i];
        hist[(gen - 1) % 10] = b;
        if (prm->autostop && gen >= 10) {
            double m = 0.0, v = 0.0;
            for (int k = 0; k < 10; ++k) m += hist[k];
            m /= 10.0;
            for (int k = 0; k < 10; ++k) v += (hist[k] - m) * (hist[k] - m);
            if (sqrt(v / 10.0) < prm->stopstd) break;
        }
    }
    int best = 0;
    for (int i = 1; i < pop; ++i) if (Pe[i] < Pe[best]) best = i;
    res->best_energy = Pe[best];
    memcpy(res->best_genes, Pg + (size_t)best * G, sizeof(double) * G);
    res->evals = P.evals;
    res->generations = gen;
    free(Pg); free(Pe); free(Ng); free(Ne);
    return ORC_OK;
}

/* Initial population alone (generation 0), for the RNG replay test. */
void orc_init_population(const orc_grid* g, const orc_params* prm, int T, int run, double* genes)
{
    orc_rng r = {{prm->seed_lo, prm->seed_hi}, prm->lig_id};
    for (int i = 0; i < prm->pop_size; ++i) init_individual(&r, g, T, run, i, genes + (size_t)i * (7 + T));
}
