/*
 * FP64 CPU oracle of the START radiative-transfer hot path
 * (Hasegawa & Umemura 2010, "START: SPH with tree-based accelerated
 * radiative transfer", Sections 2.2.1, 2.2.2, 4.1 and Appendix A).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously
 * correct statement of what the GPU path computes.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg load it; the
 * product library never links, calls or falls back to it.  It shares no
 * code, header or constant with the CUDA sources.
 *
 * Everything is FP64 (inputs are the caller's float32 values promoted
 * exactly), compiled with -ffp-contract=off so that no multiply-add is
 * fused.  Particles are addressed by their input (original) index.
 *
 * Steps, each following the paper's description:
 *   frame + Morton keys   cubic cells subdivided into 8 (Section 2.2.2)
 *   octrees               split until a cell holds at most `leaf` members
 *                         (one radiation source per cell, Section 2.2.2)
 *   moments               L = sum L_j, r = sum L_j r_j / sum L_j (Section 2.2.2;
 *                         the same form with N_rec for emitters, Eq. ssum)
 *   neighbours            particles within 2h of the target (Section 2.2.1)
 *   walk                  accept a cell when l/d <= theta_crit and its parent
 *                         was not accepted (Eqs. con1, con2)
 *   march                 tau_target = tau_up + d_tau, the upstream particle
 *                         being the neighbour with the smallest angle to the
 *                         ray (Eq. tau), d_tau = sigma dl (n_t + n_up)/2
 *   Gamma                 sum L exp(-tau) / (4 pi r^2) (Eq. solution2 with
 *                         geometric dilution, Eq. ksum / Appendix A)
 *   SPH density           rho_i = sum_j m_j W(r_ij, h_i) with the standard
 *                         cubic spline kernel (Section 2.1), over the particle
 *                         itself and its neighbours (the kernel's support)
 *   ionisation            implicit (backward Euler) hydrogen update
 *                         (Appendix A), with alpha_B on the spot or alpha_A
 *                         plus the self term k_self (Eq. kself1) in the
 *                         diffuse case (Section 4.1)
 *   H2 photodissociation  k_dis with self-shielding over the H2 column along
 *                         the same chains (Appendix B, Eqs. H2ss, NH2)
 *   spectra               blackbody point sources (Appendix A integrals) and
 *                         recombination photons in a band of width k T / h
 *                         with their photoheating (Section 4.1, Eqs. gself,
 *                         gother)
 *
 * Readings of points the paper leaves open (the same readings bind the GPU
 * path):
 *   - d in Eq. con1 is the Euclidean distance from the target to the cell
 *     cube (zero inside); the test is l*l <= theta^2 * d*d.  The root is
 *     tested by con1 alone.
 *   - A leaf that is not accepted contributes its sources individually.
 *   - The upstream particle of j for a source at r_s is the neighbour k of j
 *     that is strictly closer to r_s than j and maximises
 *     c_k = (r_s - r_j).(r_k - r_j) / |r_k - r_j| (smallest angle phi);
 *     ties go to the smaller input index.  When no neighbour is closer the
 *     chain ends with d_tau = sigma n_j |r_j - r_s|.
 *   - dl = |r_j - r_s| - |r_up - r_s| (radial difference).
 *   - n in d_tau is the neutral density n_HI.
 *   - r in the dilution is floored at 1e-6 of the root cube's side.
 *   - Single-member cells take the member's position as centroid; cells
 *     with zero luminosity take their cube centre.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_LEVELS 21
#define ORC_PI 3.14159265358979323846

typedef struct {
    double sigma_cm2;    /* photoionisation cross-section, cm^2 */
    double len_unit_cm;  /* length unit of positions, cm */
    double alpha_A;      /* recombination to all levels, cm^3/s */
    double alpha_B;      /* recombination to excited levels, cm^3/s */
    int src_leaf;        /* max sources per source-tree leaf (paper: 1) */
    int ptree_leaf;      /* max particles per particle-tree leaf */
    int diffuse;         /* 1: every particle emits recombination photons */
    int lum_kernel;      /* 1: kernel-weighted emissivity for the emitter cells'
                            luminosities (kernel_luminosities) */
    double T_rec;        /* 0: recombination photons at nu_L; else the gas
                            temperature (K) that sets their band width k T / h
                            (Section 4.1) */
} orc_params;

typedef struct {
    long n, cap;
    int *level, *leaf;
    long *first, *count, *skip;
    double *clo;   /* 3 per node: lower cube corner */
    double *edge;  /* cube edge */
    double *L;     /* summed luminosity (photons/s) */
    double *M;     /* 3 per node: summed L*r */
    float *cen;    /* 3 per node: luminosity centre rounded to float */
} otree;

typedef struct {
    orc_params p;
    long np, ns;
    float *px, *py, *pz, *h;
    float *sx, *sy, *sz;
    double *sL, *V;
    double lo[3], side;
    uint64_t *pkey, *skey;       /* keys in input order */
    long *pperm, *sperm;         /* sorted rank -> input index */
    long *prank;                 /* input index -> sorted rank */
    otree pt, st, et;
    long *nb_off, *nb_idx;
    double *eL;                  /* emitter luminosity per particle, photons/s */
} orc;

/* ------------------------------------------------------------------ */
/* small helpers                                                       */

static double d2_64(double ax, double ay, double az, double bx, double by, double bz)
{
    double dx = ax - bx, dy = ay - by, dz = az - bz;
    return (dx * dx + dy * dy) + dz * dz;
}

static void *xmalloc(size_t n) { void *p = malloc(n ? n : 1); return p; }

static void tree_free(otree *t)
{
    free(t->level); free(t->leaf); free(t->first); free(t->count); free(t->skip);
    free(t->clo); free(t->edge); free(t->L); free(t->M); free(t->cen);
    memset(t, 0, sizeof(*t));
}

static long tree_push(otree *t)
{
    if (t->n == t->cap) {
        long c = t->cap ? 2 * t->cap : 64;
        t->level = realloc(t->level, c * sizeof(int));
        t->leaf = realloc(t->leaf, c * sizeof(int));
        t->first = realloc(t->first, c * sizeof(long));
        t->count = realloc(t->count, c * sizeof(long));
        t->skip = realloc(t->skip, c * sizeof(long));
        t->clo = realloc(t->clo, 3 * c * sizeof(double));
        t->edge = realloc(t->edge, c * sizeof(double));
        t->L = realloc(t->L, c * sizeof(double));
        t->M = realloc(t->M, 3 * c * sizeof(double));
        t->cen = realloc(t->cen, 3 * c * sizeof(float));
        t->cap = c;
    }
    return t->n++;
}

/* ------------------------------------------------------------------ */
/* frame and Morton keys: cubic cells, Section 2.2.2                    */

/* Common root cube over particles and sources: lower corner = coordinate
 * minima, side = largest extent (1 when every point coincides). */
static void make_frame(orc *o)
{
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (long i = 0; i < o->np; ++i) {
        double v[3] = {o->px[i], o->py[i], o->pz[i]};
        for (int a = 0; a < 3; ++a) { if (v[a] < lo[a]) lo[a] = v[a]; if (v[a] > hi[a]) hi[a] = v[a]; }
    }
    for (long i = 0; i < o->ns; ++i) {
        double v[3] = {o->sx[i], o->sy[i], o->sz[i]};
        for (int a = 0; a < 3; ++a) { if (v[a] < lo[a]) lo[a] = v[a]; if (v[a] > hi[a]) hi[a] = v[a]; }
    }
    double side = 0.0;
    for (int a = 0; a < 3; ++a) { double e = hi[a] - lo[a]; if (e > side) side = e; }
    if (!(side > 0.0)) side = 1.0;
    for (int a = 0; a < 3; ++a) o->lo[a] = lo[a];
    o->side = side;
}

/* 21 bits per axis: q = clamp(floor((x - lo) * 2^21 / side)); the key
 * interleaves the bits from the top, x above y above z within each level. */
static uint64_t morton_key(const orc *o, float x, float y, float z)
{
    double scale = 2097152.0 / o->side;
    double v[3] = {x, y, z};
    uint64_t q[3];
    for (int a = 0; a < 3; ++a) {
        double t = floor((v[a] - o->lo[a]) * scale);
        if (t < 0.0) t = 0.0;
        if (t > 2097151.0) t = 2097151.0;
        q[a] = (uint64_t)t;
    }
    uint64_t key = 0;
    for (int b = ORC_LEVELS - 1; b >= 0; --b)
        key = (key << 3) | (((q[0] >> b) & 1u) << 2) | (((q[1] >> b) & 1u) << 1) | ((q[2] >> b) & 1u);
    return key;
}

static const uint64_t *g_sort_keys;
static int cmp_key_index(const void *a, const void *b)
{
    long i = *(const long *)a, j = *(const long *)b;
    uint64_t ki = g_sort_keys[i], kj = g_sort_keys[j];
    if (ki < kj) return -1;
    if (ki > kj) return 1;
    return (i > j) - (i < j);
}

/* stable order by (key, input index) */
static void sort_by_key(const uint64_t *key, long n, long *perm)
{
    for (long i = 0; i < n; ++i) perm[i] = i;
    g_sort_keys = key;
    qsort(perm, n, sizeof(long), cmp_key_index);
}

/* ------------------------------------------------------------------ */
/* octree: a cell is split into its non-empty octants while it holds
 * more than `leaf` members and is above the finest level.              */

static int digit_at(uint64_t key, int level)   /* octant digit of level 1..21 */
{
    return (int)((key >> (3 * (ORC_LEVELS - level))) & 7u);
}

static long build_node(const orc *o, otree *t, const uint64_t *skeys, int level,
                       long first, long count, long leaf)
{
    long id = tree_push(t);
    t->level[id] = level;
    t->first[id] = first;
    t->count[id] = count;
    /* cube of this cell from the key prefix of its first member */
    uint64_t prefix = level ? (skeys[first] >> (3 * (ORC_LEVELS - level))) : 0;
    uint64_t ix[3] = {0, 0, 0};
    for (int m = 0; m < level; ++m) {
        ix[0] |= ((prefix >> (3 * m + 2)) & 1u) << m;
        ix[1] |= ((prefix >> (3 * m + 1)) & 1u) << m;
        ix[2] |= ((prefix >> (3 * m)) & 1u) << m;
    }
    double l = ldexp(o->side, -level);
    t->edge[id] = l;
    for (int a = 0; a < 3; ++a) t->clo[3 * id + a] = o->lo[a] + (double)ix[a] * l;
    int split = count > leaf && level < ORC_LEVELS;
    t->leaf[id] = !split;
    if (split) {
        long i = first, end = first + count;
        while (i < end) {
            int d = digit_at(skeys[i], level + 1);
            long j = i;
            while (j < end && digit_at(skeys[j], level + 1) == d) ++j;
            build_node(o, t, skeys, level + 1, i, j - i, leaf);
            i = j;
        }
    }
    t->skip[id] = t->n;
    return id;
}

static void build_tree(const orc *o, otree *t, const uint64_t *skeys, long n, long leaf)
{
    tree_free(t);
    if (n > 0) build_node(o, t, skeys, 0, 0, n, leaf);
}

/* Luminosity moments (Section 2.2.2 / Eq. ssum): a leaf sums its members in
 * sorted order, an inner cell sums its children in octant order. */
static void moments_node(otree *t, long n, const long *perm, const float *x, const float *y,
                         const float *z, const double *L)
{
    double S = 0.0, Mx = 0.0, My = 0.0, Mz = 0.0;
    if (t->leaf[n]) {
        for (long r = t->first[n]; r < t->first[n] + t->count[n]; ++r) {
            long j = perm[r];
            S += L[j];
            Mx += L[j] * (double)x[j];
            My += L[j] * (double)y[j];
            Mz += L[j] * (double)z[j];
        }
    } else {
        for (long c = n + 1; c < t->skip[n]; c = t->skip[c]) {
            moments_node(t, c, perm, x, y, z, L);
            S += t->L[c];
            Mx += t->M[3 * c];
            My += t->M[3 * c + 1];
            Mz += t->M[3 * c + 2];
        }
    }
    t->L[n] = S;
    t->M[3 * n] = Mx; t->M[3 * n + 1] = My; t->M[3 * n + 2] = Mz;
    if (t->count[n] == 1) {
        long j = perm[t->first[n]];
        t->cen[3 * n] = x[j]; t->cen[3 * n + 1] = y[j]; t->cen[3 * n + 2] = z[j];
    } else if (S > 0.0) {
        t->cen[3 * n] = (float)(Mx / S);
        t->cen[3 * n + 1] = (float)(My / S);
        t->cen[3 * n + 2] = (float)(Mz / S);
    } else {
        for (int a = 0; a < 3; ++a)
            t->cen[3 * n + a] = (float)(t->clo[3 * n + a] + 0.5 * t->edge[n]);
    }
}

/* ------------------------------------------------------------------ */
/* neighbours: N(i) = { k != i : |r_k - r_i| < 2 h_i }, found through the
 * particle octree (Section 2.2.2 reuses the gravity tree).              */

typedef struct { long *v; long n, cap; } lvec;
static void lvec_push(lvec *a, long x)
{
    if (a->n == a->cap) { a->cap = a->cap ? 2 * a->cap : 64; a->v = realloc(a->v, a->cap * sizeof(long)); }
    a->v[a->n++] = x;
}

static double box_d2(const otree *t, long n, double px, double py, double pz)
{
    double l = t->edge[n];
    double p[3] = {px, py, pz};
    double d[3];
    for (int a = 0; a < 3; ++a) {
        double lo = t->clo[3 * n + a], hi = lo + l;
        d[a] = 0.0;
        if (p[a] < lo) d[a] = lo - p[a];
        else if (p[a] > hi) d[a] = p[a] - hi;
    }
    return (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
}

static void nb_collect(const orc *o, long n, long i, lvec *out)
{
    const otree *t = &o->pt;
    double px = o->px[i], py = o->py[i], pz = o->pz[i];
    double two_h = 2.0 * (double)o->h[i];
    double r2 = two_h * two_h;
    /* cells are visited with a small slack: members can sit a rounding
     * error outside their cube; the member test below is exact. */
    double slack = 1e-9 * o->side;
    double bd = sqrt(box_d2(t, n, px, py, pz));
    if (bd > two_h + slack) return;
    if (t->leaf[n]) {
        for (long r = t->first[n]; r < t->first[n] + t->count[n]; ++r) {
            long k = o->pperm[r];
            if (k == i) continue;
            if (d2_64(o->px[k], o->py[k], o->pz[k], px, py, pz) < r2) lvec_push(out, k);
        }
        return;
    }
    for (long c = n + 1; c < t->skip[n]; c = t->skip[c]) nb_collect(o, c, i, out);
}

static int cmp_long(const void *a, const void *b)
{
    long x = *(const long *)a, y = *(const long *)b;
    return (x > y) - (x < y);
}

static void build_neighbours(orc *o)
{
    free(o->nb_off); free(o->nb_idx);
    o->nb_off = xmalloc((o->np + 1) * sizeof(long));
    lvec *rows = calloc(o->np ? o->np : 1, sizeof(lvec));
#pragma omp parallel for schedule(dynamic, 256)
    for (long i = 0; i < o->np; ++i) {
        if (o->pt.n) nb_collect(o, 0, i, &rows[i]);
        qsort(rows[i].v, rows[i].n, sizeof(long), cmp_long);
    }
    long tot = 0;
    for (long i = 0; i < o->np; ++i) { o->nb_off[i] = tot; tot += rows[i].n; }
    o->nb_off[o->np] = tot;
    o->nb_idx = xmalloc(tot * sizeof(long));
    for (long i = 0; i < o->np; ++i) {
        if (rows[i].n) memcpy(o->nb_idx + o->nb_off[i], rows[i].v, rows[i].n * sizeof(long));
        free(rows[i].v);
    }
    free(rows);
}

/* ------------------------------------------------------------------ */
/* walk: Eqs. con1 / con2                                               */

static int accept_cell(const otree *t, long n, double px, double py, double pz, double th2)
{
    double l = t->edge[n];
    return l * l <= th2 * box_d2(t, n, px, py, pz);
}

/* Entries: node id >= 0 for an accepted cell, -(1 + sorted rank) for an
 * individual member of a leaf that was not accepted. */
static void walk_node(const otree *t, long n, double px, double py, double pz, double th2,
                      long self_rank, lvec *out)
{
    if (accept_cell(t, n, px, py, pz, th2)) { lvec_push(out, n); return; }
    if (t->leaf[n]) {
        for (long r = t->first[n]; r < t->first[n] + t->count[n]; ++r)
            if (r != self_rank) lvec_push(out, -(1 + r));
        return;
    }
    for (long c = n + 1; c < t->skip[n]; c = t->skip[c])
        walk_node(t, c, px, py, pz, th2, self_rank, out);
}

/* ------------------------------------------------------------------ */
/* march: Eq. tau and the trapezoidal d_tau (Section 2.2.1)             */

/* Column of the density field `dens` from rs to particle i along the chain,
 * times `scale`: scale = sigma * len_unit gives tau (Eq. tau, dens = n_HI),
 * scale = len_unit gives a column density in cm^-2 (Eq. NH2, dens = n_H2). */
static double march_column(const orc *o, long i, const double rs[3], const float *dens,
                           double sig, long *hops, lvec *chain)
{
    const float *nHI = dens;
    long j = i;
    double tau = 0.0;
    long nh = 0;
    for (;;) {
        double jx = o->px[j], jy = o->py[j], jz = o->pz[j];
        double Dj = d2_64(jx, jy, jz, rs[0], rs[1], rs[2]);
        double bx = rs[0] - jx, by = rs[1] - jy, bz = rs[2] - jz;
        long best = -1;
        double cbest = 0.0;
        ++nh;
        for (long e = o->nb_off[j]; e < o->nb_off[j + 1]; ++e) {
            long k = o->nb_idx[e];
            double kx = o->px[k], ky = o->py[k], kz = o->pz[k];
            double Dk = d2_64(kx, ky, kz, rs[0], rs[1], rs[2]);
            if (!(Dk < Dj)) continue;
            double ax = kx - jx, ay = ky - jy, az = kz - jz;
            double dot = (bx * ax + by * ay) + bz * az;
            double c = dot / sqrt(d2_64(kx, ky, kz, jx, jy, jz));
            if (best < 0 || c > cbest || (c == cbest && k < best)) { best = k; cbest = c; }
        }
        if (chain) lvec_push(chain, j);
        if (best < 0) {
            tau += sig * (double)nHI[j] * sqrt(Dj);
            break;
        }
        double Db = d2_64(o->px[best], o->py[best], o->pz[best], rs[0], rs[1], rs[2]);
        double dl = sqrt(Dj) - sqrt(Db);
        tau += sig * 0.5 * ((double)nHI[j] + (double)nHI[best]) * dl;
        j = best;
        if (nh > o->np + 1) break;   /* cannot happen: distances strictly decrease */
    }
    if (hops) *hops += nh;
    return tau;
}

static double march(const orc *o, long i, const double rs[3], const float *nHI, long *hops,
                    lvec *chain)
{
    /* per length unit per cm^-3 */
    return march_column(o, i, rs, nHI, o->p.sigma_cm2 * o->p.len_unit_cm, hops, chain);
}

/* ------------------------------------------------------------------ */
/* public API                                                          */

orc *orc_create(const orc_params *p)
{
    orc *o = calloc(1, sizeof(orc));
    o->p = *p;
    if (o->p.src_leaf < 1) o->p.src_leaf = 1;
    if (o->p.ptree_leaf < 1) o->p.ptree_leaf = 8;
    return o;
}

void orc_destroy(orc *o)
{
    if (!o) return;
    free(o->px); free(o->py); free(o->pz); free(o->h);
    free(o->sx); free(o->sy); free(o->sz); free(o->sL); free(o->V);
    free(o->pkey); free(o->skey); free(o->pperm); free(o->sperm); free(o->prank);
    tree_free(&o->pt); tree_free(&o->st); tree_free(&o->et);
    free(o->nb_off); free(o->nb_idx); free(o->eL);
    free(o);
}

int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* pos/src_pos are SoA (3 x n) float32, h float32, src_L photons/s, V in
 * length-unit^3 (may be NULL when not diffuse). */
int orc_build(orc *o, const float *pos, const float *h, long np, const float *spos,
              const double *sL, long ns, const double *V)
{
    if (np < 0 || ns < 0) return -1;
    o->np = np; o->ns = ns;
    size_t fp = (np ? np : 1) * sizeof(float), fs = (ns ? ns : 1) * sizeof(float);
    o->px = realloc(o->px, fp); o->py = realloc(o->py, fp); o->pz = realloc(o->pz, fp);
    o->h = realloc(o->h, fp);
    o->sx = realloc(o->sx, fs); o->sy = realloc(o->sy, fs); o->sz = realloc(o->sz, fs);
    o->sL = realloc(o->sL, (ns ? ns : 1) * sizeof(double));
    o->V = realloc(o->V, (np ? np : 1) * sizeof(double));
    memcpy(o->px, pos, np * sizeof(float));
    memcpy(o->py, pos + np, np * sizeof(float));
    memcpy(o->pz, pos + 2 * np, np * sizeof(float));
    memcpy(o->h, h, np * sizeof(float));
    memcpy(o->sx, spos, ns * sizeof(float));
    memcpy(o->sy, spos + ns, ns * sizeof(float));
    memcpy(o->sz, spos + 2 * ns, ns * sizeof(float));
    memcpy(o->sL, sL, ns * sizeof(double));
    for (long i = 0; i < np; ++i) o->V[i] = V ? V[i] : 0.0;

    make_frame(o);
    o->pkey = realloc(o->pkey, (np ? np : 1) * sizeof(uint64_t));
    o->skey = realloc(o->skey, (ns ? ns : 1) * sizeof(uint64_t));
    for (long i = 0; i < np; ++i) o->pkey[i] = morton_key(o, o->px[i], o->py[i], o->pz[i]);
    for (long i = 0; i < ns; ++i) o->skey[i] = morton_key(o, o->sx[i], o->sy[i], o->sz[i]);
    o->pperm = realloc(o->pperm, (np ? np : 1) * sizeof(long));
    o->sperm = realloc(o->sperm, (ns ? ns : 1) * sizeof(long));
    o->prank = realloc(o->prank, (np ? np : 1) * sizeof(long));
    sort_by_key(o->pkey, np, o->pperm);
    sort_by_key(o->skey, ns, o->sperm);
    for (long r = 0; r < np; ++r) o->prank[o->pperm[r]] = r;

    uint64_t *pks = xmalloc((np ? np : 1) * sizeof(uint64_t));
    uint64_t *sks = xmalloc((ns ? ns : 1) * sizeof(uint64_t));
    for (long r = 0; r < np; ++r) pks[r] = o->pkey[o->pperm[r]];
    for (long r = 0; r < ns; ++r) sks[r] = o->skey[o->sperm[r]];
    build_tree(o, &o->pt, pks, np, o->p.ptree_leaf);
    build_tree(o, &o->st, sks, ns, o->p.src_leaf);
    if (o->p.diffuse) build_tree(o, &o->et, pks, np, o->p.src_leaf);
    else tree_free(&o->et);
    free(pks); free(sks);
    if (o->st.n) moments_node(&o->st, 0, o->sperm, o->sx, o->sy, o->sz, o->sL);
    build_neighbours(o);
    free(o->eL);
    o->eL = calloc(np ? np : 1, sizeof(double));
    if (o->et.n) moments_node(&o->et, 0, o->pperm, o->px, o->py, o->pz, o->eL);
    return 0;
}

void orc_frame(const orc *o, double out[4])
{
    out[0] = o->lo[0]; out[1] = o->lo[1]; out[2] = o->lo[2]; out[3] = o->side;
}

/* which: 0 particles, 1 sources */
void orc_keys(const orc *o, int which, uint64_t *out)
{
    if (which == 0) memcpy(out, o->pkey, o->np * sizeof(uint64_t));
    else memcpy(out, o->skey, o->ns * sizeof(uint64_t));
}

void orc_perm(const orc *o, int which, long *out)
{
    if (which == 0) memcpy(out, o->pperm, o->np * sizeof(long));
    else memcpy(out, o->sperm, o->ns * sizeof(long));
}

static const otree *pick_tree(const orc *o, int which)
{
    return which == 0 ? &o->pt : which == 1 ? &o->st : &o->et;
}

/* which: 0 particle tree, 1 source tree, 2 emitter tree */
long orc_tree_size(const orc *o, int which) { return pick_tree(o, which)->n; }

void orc_tree_get(const orc *o, int which, int *level, long *first, long *count, long *skip,
                  int *leaf, double *cube4, double *L, double *M3, float *cen3)
{
    const otree *t = pick_tree(o, which);
    for (long n = 0; n < t->n; ++n) {
        if (level) level[n] = t->level[n];
        if (first) first[n] = t->first[n];
        if (count) count[n] = t->count[n];
        if (skip) skip[n] = t->skip[n];
        if (leaf) leaf[n] = t->leaf[n];
        if (cube4) {
            cube4[4 * n] = t->clo[3 * n]; cube4[4 * n + 1] = t->clo[3 * n + 1];
            cube4[4 * n + 2] = t->clo[3 * n + 2]; cube4[4 * n + 3] = t->edge[n];
        }
        if (L) L[n] = t->L[n];
        if (M3) { M3[3 * n] = t->M[3 * n]; M3[3 * n + 1] = t->M[3 * n + 1]; M3[3 * n + 2] = t->M[3 * n + 2]; }
        if (cen3) { cen3[3 * n] = t->cen[3 * n]; cen3[3 * n + 1] = t->cen[3 * n + 1]; cen3[3 * n + 2] = t->cen[3 * n + 2]; }
    }
}

long orc_nbr_total(const orc *o) { return o->np ? o->nb_off[o->np] : 0; }

void orc_nbr_get(const orc *o, long *off, long *idx)
{
    memcpy(off, o->nb_off, (o->np + 1) * sizeof(long));
    memcpy(idx, o->nb_idx, orc_nbr_total(o) * sizeof(long));
}

/* The kernel-weighted form of a virtual source's luminosity (Section 2.2.2
 * offers L = sum_j L_j W(r - r_j) / sum_j W(r - r_j) as an alternative).
 * Reading: the weighted quantity is the emissivity L_j / V_j (V_j = m_j /
 * rho_j, the particle's volume), so the weighted mean is an emissivity and
 * the cell's volume l^3 turns it into the cell's luminosity:
 *   L_cell = l^3 sum_j (L_j / V_j) W(|r_c - r_j|, l) / sum_j W(|r_c - r_j|, l)
 * over the cell's members j, r_c the cell's luminosity centre as stored
 * (float32), W the cubic spline with smoothing length h = l (its support 2l
 * reaches every member from any point of the cell), for every cell of more
 * than one member; a single-member cell keeps its member's luminosity.  A
 * uniform emissivity gives l^3 times it, the summed luminosity of a cell
 * that its members fill.  Emitter tree only (its members are SPH particles
 * with volumes); the centres keep the luminosity-weighted form. */
double orc_spline_w(double r, double h);

static void kernel_luminosities(orc *o)
{
    otree *t = &o->et;
    for (long n = 0; n < t->n; ++n) {
        if (t->count[n] < 2) continue;
        double l = t->edge[n];
        double cx = t->cen[3 * n], cy = t->cen[3 * n + 1], cz = t->cen[3 * n + 2];
        double sw = 0.0, se = 0.0;
        for (long r = t->first[n]; r < t->first[n] + t->count[n]; ++r) {
            long j = o->pperm[r];
            double d = sqrt(d2_64(o->px[j], o->py[j], o->pz[j], cx, cy, cz));
            double w = orc_spline_w(d, l);
            sw += w;
            se += (o->eL[j] / o->V[j]) * w;
        }
        if (sw > 0.0) t->L[n] = l * l * l * (se / sw);
    }
}

/* Recombination emitters (Section 4.1): N_rec,j = alpha_1 n_e n_p V_j with
 * n_e = n_p = x n_H (hydrogen only), alpha_1 = alpha_A - alpha_B; then the
 * emitter tree's moments.  y is the neutral fraction in input order. */
void orc_set_emitters(orc *o, const double *y, const float *nH)
{
    double a1 = o->p.alpha_A - o->p.alpha_B;
    double lu3 = o->p.len_unit_cm * o->p.len_unit_cm * o->p.len_unit_cm;
    for (long i = 0; i < o->np; ++i) {
        double ne = (1.0 - y[i]) * (double)nH[i];
        o->eL[i] = a1 * ne * ne * (o->V[i] * lu3);
    }
    if (o->et.n) moments_node(&o->et, 0, o->pperm, o->px, o->py, o->pz, o->eL);
    if (o->et.n && o->p.lum_kernel) kernel_luminosities(o);
}

double orc_emitter_L(const orc *o, long i) { return o->eL[i]; }

/* Interaction list of one target (input index) on tree `which` (1 sources,
 * 2 emitters).  Returns the number of entries; writes at most cap. */
long orc_list(const orc *o, int which, float theta, long target, long *out, long cap)
{
    const otree *t = pick_tree(o, which);
    lvec v = {0};
    double th = theta;
    if (t->n) walk_node(t, 0, o->px[target], o->py[target], o->pz[target], th * th,
                        which == 2 ? o->prank[target] : -1, &v);
    long n = v.n;
    for (long e = 0; e < n && e < cap; ++e) out[e] = v.v[e];
    free(v.v);
    return n;
}

/* Whole-row checksums of the interaction lists (all trees walked by a
 * solve: the sources, then in the diffuse case the emitters), for comparing
 * them with a list computed elsewhere without copying every entry.  Each
 * entry is encoded as an unsigned 32-bit word -- the cell's node id, or
 * 0x80000000 | sorted rank for a member of a leaf that was not accepted,
 * with 0x40000000 added on the emitter tree -- and fed to the 64-bit FNV-1a
 * hash (offset basis 14695981039346656037, prime 1099511628211) as four
 * bytes, least significant first, in walk order.  count = row length. */
void orc_list_hashes(const orc *o, float theta, const long *targets, long nt, uint64_t *hash,
                     long *count)
{
    long n = targets ? nt : o->np;
    double th = theta;
#pragma omp parallel for schedule(dynamic, 64)
    for (long t = 0; t < n; ++t) {
        long i = targets ? targets[t] : t;
        uint64_t h = 14695981039346656037ull;
        long len = 0;
        for (int which = 1; which <= (o->p.diffuse ? 2 : 1); ++which) {
            const otree *tr = pick_tree(o, which);
            if (!tr->n) continue;
            lvec v = {0};
            walk_node(tr, 0, o->px[i], o->py[i], o->pz[i], th * th,
                      which == 2 ? o->prank[i] : -1, &v);
            for (long e = 0; e < v.n; ++e) {
                long ent = v.v[e];
                uint32_t w = ent >= 0 ? (uint32_t)ent : (0x80000000u | (uint32_t)(-ent - 1));
                if (which == 2) w |= 0x40000000u;
                for (int b = 0; b < 4; ++b) {
                    h ^= (w >> (8 * b)) & 0xffu;
                    h *= 1099511628211ull;
                }
            }
            len += v.n;
            free(v.v);
        }
        hash[t] = h;
        if (count) count[t] = len;
    }
}

/* Optical depth from a source at rs to particle `target`; the visited chain
 * (input indices, target first) goes to chain_out when given. */
double orc_march(const orc *o, long target, const float rs32[3], const float *nHI, long *hops,
                 long *chain_out, long cap, long *chain_len)
{
    double rs[3] = {rs32[0], rs32[1], rs32[2]};
    lvec ch = {0};
    long nh = 0;
    double tau = march(o, target, rs, nHI, &nh, chain_out ? &ch : NULL);
    if (hops) *hops = nh;
    if (chain_out) {
        for (long e = 0; e < ch.n && e < cap; ++e) chain_out[e] = ch.v[e];
        if (chain_len) *chain_len = ch.n;
    }
    free(ch.v);
    return tau;
}

static void bb_integrals(double tau, double a, double *f_ion, double *f_heat);
static void band_integrals(double tau, double D, double *r_ion, double *r_heat);

/* Sum over the interaction list of target i on one tree, in walk order.
 * spec 0: photons at nu_L, L e^-tau / (4 pi r^2), no heating; spec 1:
 * blackbody with a = h nu_L / (k T_eff), L F_ion(tau) / (4 pi r^2) and the
 * heating factor L F_heat(tau) / (4 pi r^2); spec 2: the recombination band of
 * width D = k T_rec / (h nu_L), the same with R_ion and R_heat.  Returns the
 * Gamma sum and adds the heating factors to *heat. */
static double tree_sum(const orc *o, int which, long i, double th, const float *nHI, int spec,
                       double par, double *heat, long long *rays, long long *hops)
{
    const otree *t = pick_tree(o, which);
    if (!t->n) return 0.0;
    lvec v = {0};
    walk_node(t, 0, o->px[i], o->py[i], o->pz[i], th * th, which == 2 ? o->prank[i] : -1, &v);
    double lu = o->p.len_unit_cm;
    double rfloor = 1e-6 * o->side;
    double g = 0.0;
    for (long e = 0; e < v.n; ++e) {
        double rs[3], L;
        long ent = v.v[e];
        if (ent >= 0) {
            rs[0] = t->cen[3 * ent]; rs[1] = t->cen[3 * ent + 1]; rs[2] = t->cen[3 * ent + 2];
            L = t->L[ent];
        } else {
            long r = -ent - 1;
            if (which == 1) {
                long j = o->sperm[r];
                rs[0] = o->sx[j]; rs[1] = o->sy[j]; rs[2] = o->sz[j];
                L = o->sL[j];
            } else {
                long j = o->pperm[r];
                rs[0] = o->px[j]; rs[1] = o->py[j]; rs[2] = o->pz[j];
                L = o->eL[j];
            }
        }
        long nh = 0;
        double tau = march(o, i, rs, nHI, &nh, NULL);
        double r2 = d2_64(o->px[i], o->py[i], o->pz[i], rs[0], rs[1], rs[2]);
        if (r2 < rfloor * rfloor) r2 = rfloor * rfloor;
        if (spec == 0) {
            g += L * exp(-tau) / (4.0 * ORC_PI * r2 * lu * lu);
        } else {
            double fi, fh;
            if (spec == 1) bb_integrals(tau, par, &fi, &fh);
            else band_integrals(tau, par, &fi, &fh);
            double flux = L / (4.0 * ORC_PI * r2 * lu * lu);
            g += flux * fi;
            *heat += flux * fh;
        }
        *rays += 1;
        *hops += nh;
    }
    free(v.v);
    return g;
}

/* Gamma of one target from one tree: sum over its list in walk order. */
static double gamma_tree(const orc *o, int which, long i, double th, const float *nHI,
                         long long *rays, long long *hops)
{
    double unused = 0.0;
    return tree_sum(o, which, i, th, nHI, 0, 0.0, &unused, rays, hops);
}

/* Photoionisation rate Gamma (photons cm^-2 s^-1) at the given targets
 * (input indices; NULL = all particles in order).  nHI is in input order.
 * In the diffuse case the emitter tree (after orc_set_emitters) adds the
 * recombination photons of every other particle.  stats = {rays, hops}. */
int orc_gamma(const orc *o, const float *nHI, float theta, const long *targets, long nt,
              double *gamma_out, long long *stats)
{
    long n = targets ? nt : o->np;
    long long rays = 0, hops = 0;
    double th = theta;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : rays, hops)
    for (long t = 0; t < n; ++t) {
        long i = targets ? targets[t] : t;
        long long r = 0, hcount = 0;
        double g = gamma_tree(o, 1, i, th, nHI, &r, &hcount);
        if (o->p.diffuse) g += gamma_tree(o, 2, i, th, nHI, &r, &hcount);
        gamma_out[t] = g;
        rays += r;
        hops += hcount;
    }
    if (stats) { stats[0] = rays; stats[1] = hops; }
    return 0;
}

#define ORC_HNU_L_ERG (13.6 * 1.602176634e-12)   /* h nu_L = 13.6 eV */
#define ORC_KB_ERG 1.380649e-16                  /* Boltzmann constant, erg/K */

/* Self terms of a particle per neutral atom, from its state (y0, n_H) and
 * volume V: the photoionisation rate k_self of Eq. kself1 in its reduced form
 * and the photoheating rate of Eq. gself divided by n_HI.  With
 * n_e = n_p = x n_H, tau_s = sigma n_HI R, R = (3V/4pi)^(1/3) and
 * phi(t) = (1 - e^-t)/t (the division by n_HI taken inside phi, so that a
 * fully ionised particle is regular):
 *   photons at nu_L (T_rec = 0): k_self = alpha_1 n_e n_p sigma R phi(tau_s),
 *     no heating;
 *   the band 1 <= u <= 1 + D, D = k T_rec / (h nu_L), sigma_nu = sigma u^-3:
 *     k_self = alpha_1 n_e n_p sigma R (1/D) int u^-3 phi(tau_s u^-3) du
 *     heat   = alpha_1 n_e n_p sigma R h nu_L (1/D) int (u-1) u^-3 phi(tau_s u^-3) du
 *     by composite Simpson with 512 intervals. */
static void self_terms_a1(const orc *o, long i, double nh, double y0, double a1,
                          double *k_self, double *h_self)
{
    double sig = o->p.sigma_cm2;
    double x0 = 1.0 - y0;
    double R = cbrt(3.0 * o->V[i] / (4.0 * ORC_PI)) * o->p.len_unit_cm;
    double ts = sig * (y0 * nh) * R;
    if (o->p.T_rec <= 0.0) {
        double phi = ts > 0.0 ? -expm1(-ts) / ts : 1.0;
        *k_self = a1 * x0 * x0 * nh * nh * sig * R * phi;
        *h_self = 0.0;
        return;
    }
    double D = ORC_KB_ERG * o->p.T_rec / ORC_HNU_L_ERG;
    const int n = 512;
    double du = D / n, si = 0.0, sh = 0.0;
    for (int k = 0; k <= n; ++k) {
        double u = 1.0 + k * du;
        double wgt = (k == 0 || k == n) ? 1.0 : ((k & 1) ? 4.0 : 2.0);
        double u3 = 1.0 / (u * u * u);
        double t = ts * u3;
        double phi = t > 0.0 ? -expm1(-t) / t : 1.0;
        si += wgt * u3 * phi;
        sh += wgt * (u - 1.0) * u3 * phi;
    }
    double pre = a1 * x0 * x0 * nh * nh * sig * R;
    *k_self = pre * (si * du / (3.0 * D));
    *h_self = pre * ORC_HNU_L_ERG * (sh * du / (3.0 * D));
}

static void self_terms(const orc *o, long i, double nh, double y0, double *k_self,
                       double *h_self)
{
    self_terms_a1(o, i, nh, y0, o->p.alpha_A - o->p.alpha_B, k_self, h_self);
}

double orc_rate(int which, double T);

/* Self terms of particles [0, n) (input order, diffuse case): k_self and the
 * self photoheating, both per neutral atom; with temperatures T (may be
 * NULL) alpha_1 = alpha_A(T) - alpha_B(T) of the rate fits below. */
void orc_self_terms(const orc *o, const float *nH, const double *y0, long n, double *k_self,
                    double *h_self)
{
    for (long i = 0; i < n; ++i) self_terms(o, i, (double)nH[i], y0[i], &k_self[i], &h_self[i]);
}

void orc_self_terms_T(const orc *o, const float *nH, const double *y0, const double *T, long n,
                      double *k_self, double *h_self)
{
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) {
        double a1 = T ? orc_rate(0, T[i]) - orc_rate(1, T[i]) : o->p.alpha_A - o->p.alpha_B;
        self_terms_a1(o, i, (double)nH[i], y0[i], a1, &k_self[i], &h_self[i]);
    }
}

/* Implicit hydrogen update over dt (Appendix A), hydrogen only, isothermal:
 * dy/dt = -k y + alpha n_H (1 - y)^2 for the neutral fraction y, solved by
 * one backward-Euler step.  k = sigma Gamma, plus in the diffuse case the
 * self term of Eq. kself1 per neutral atom (self_terms), taken from the
 * step-start state.  Writes y1 and the float32 neutral density y1 n_H. */
void orc_ionize(const orc *o, const double *gamma, const float *nH, const double *y0, double dt,
                long n, double *y1, float *nHI_out)
{
    double alpha = o->p.diffuse ? o->p.alpha_A : o->p.alpha_B;
    double sig = o->p.sigma_cm2;
    for (long i = 0; i < n; ++i) {
        double nh = nH[i];
        double k = sig * gamma[i];
        if (o->p.diffuse) {
            double ks, hs;
            self_terms(o, i, nh, y0[i], &ks, &hs);
            k += ks;
        }
        /* y1 - y0 = dt (-k y1 + alpha n_H (1 - y1)^2): A y1^2 - b y1 + c = 0 */
        double A = alpha * nh * dt, K = k * dt;
        double b = 2.0 * A + K + 1.0, c = A + y0[i];
        double disc = (K + 1.0) * (K + 1.0) + 4.0 * A * (K + 1.0 - y0[i]);
        double y = 2.0 * c / (b + sqrt(disc));
        y1[i] = y;
        if (nHI_out) nHI_out[i] = (float)(y * nh);
    }
}

/* ------------------------------------------------------------------ */
/* SPH density (Section 2.1)                                           */

/* The standard cubic spline of SPH (Monaghan 1992) in three dimensions,
 * support 2h:  W = 1/(pi h^3) * (1 - 3/2 q^2 + 3/4 q^3)  for 0 <= q < 1,
 *                  1/(pi h^3) * (2 - q)^3 / 4             for 1 <= q < 2,
 *                  0 beyond, with q = r / h. */
double orc_spline_w(double r, double h)
{
    double q = r / h;
    double norm = 1.0 / (ORC_PI * h * h * h);
    if (q < 1.0) return norm * (1.0 - 1.5 * q * q + 0.75 * q * q * q);
    if (q < 2.0) {
        double t = 2.0 - q;
        return norm * 0.25 * t * t * t;
    }
    return 0.0;
}

/* rho_i = sum_j m_j W(|r_i - r_j|, h_i) (Section 2.1): the particle itself
 * (r = 0) and its neighbours, which are exactly the particles inside the
 * kernel's support 2 h_i.  mass and rho in input order. */
void orc_sph_density(const orc *o, const double *mass, double *rho)
{
    for (long i = 0; i < o->np; ++i) {
        double hi = o->h[i];
        double s = mass[i] * orc_spline_w(0.0, hi);
        for (long e = o->nb_off[i]; e < o->nb_off[i + 1]; ++e) {
            long k = o->nb_idx[e];
            double r = sqrt(d2_64(o->px[k], o->py[k], o->pz[k], o->px[i], o->py[i], o->pz[i]));
            s += mass[k] * orc_spline_w(r, hi);
        }
        rho[i] = s;
    }
}

/* ------------------------------------------------------------------ */
/* H2 photodissociation (Appendix B)                                   */

/* Self-shielding function f_sh(x) = 1 for x <= 1, x^(-3/4) beyond, with
 * x = N_H2 / 1e14 cm^-2 (Eq. H2ss). */
double orc_h2_fsh(double x)
{
    return x <= 1.0 ? 1.0 : pow(x, -0.75);
}

/* k_dis (s^-1) at the given targets (input indices; NULL = all): over the
 * interaction list of the point-source tree, sum 1.13e8 F_LW,0 f_sh(N_H2 /
 * 1e14 cm^-2) with F_LW,0 = kappa L / (4 pi r^2) (no absorption by H atoms
 * in the Lyman-Werner band) and N_H2 = N_H2,up + dl (n_H2,up + n_H2,tar)/2
 * along the same chain as tau (Eq. NH2), closed by n_H2 |r_j - r_s| at the
 * chain end.  kappa converts a source's ionising photon rate into its LW
 * specific luminosity.  nH2 in input order; stats = {rays, hops}. */
int orc_h2_dissociation(const orc *o, const float *nH2, float theta, double kappa,
                        const long *targets, long nt, double *out, long long *stats)
{
    long n = targets ? nt : o->np;
    long long rays = 0, hops = 0;
    double th = theta;
    const otree *t = &o->st;
    double lu = o->p.len_unit_cm;
    double rfloor = 1e-6 * o->side;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : rays, hops)
    for (long q = 0; q < n; ++q) {
        long i = targets ? targets[q] : q;
        double k = 0.0;
        if (t->n) {
            lvec v = {0};
            walk_node(t, 0, o->px[i], o->py[i], o->pz[i], th * th, -1, &v);
            for (long e = 0; e < v.n; ++e) {
                double rs[3], L;
                long ent = v.v[e];
                if (ent >= 0) {
                    rs[0] = t->cen[3 * ent]; rs[1] = t->cen[3 * ent + 1]; rs[2] = t->cen[3 * ent + 2];
                    L = t->L[ent];
                } else {
                    long j = o->sperm[-ent - 1];
                    rs[0] = o->sx[j]; rs[1] = o->sy[j]; rs[2] = o->sz[j];
                    L = o->sL[j];
                }
                long nh = 0;
                double col = march_column(o, i, rs, nH2, lu, &nh, NULL);
                double r2 = d2_64(o->px[i], o->py[i], o->pz[i], rs[0], rs[1], rs[2]);
                if (r2 < rfloor * rfloor) r2 = rfloor * rfloor;
                double F = kappa * L / (4.0 * ORC_PI * r2 * lu * lu);
                k += 1.13e8 * F * orc_h2_fsh(col / 1e14);
                rays += 1;
                hops += nh;
            }
            free(v.v);
        }
        out[q] = k;
    }
    if (stats) { stats[0] = rays; stats[1] = hops; }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Multi-frequency point sources: photoionisation and photoheating      */
/* (Appendix A integrals with blackbody sources as in Section 3.1.1)    */

/* The spectral integrals of one ray with Lyman-limit optical depth tau, per
 * ionising photon emitted: with u = nu / nu_L, the blackbody photon spectrum
 * w(u) = u^2 / (e^(a u) - 1), a = h nu_L / (k T_eff), normalised over u >= 1,
 * and the hydrogenic cross-section sigma_nu = sigma_L u^-3 (so tau_nu = tau u^-3):
 *   F_ion(tau)  = int w u^-3 e^(-tau u^-3) du / int w du
 *   F_heat(tau) = int w u^-3 (u - 1) e^(-tau u^-3) du / int w du
 * by composite Simpson over [1, 1 + 60/a] (the spectrum beyond is below e^-60
 * of its peak) with 4096 intervals. */
static void bb_integrals(double tau, double a, double *f_ion, double *f_heat)
{
    const int n = 4096;
    double umax = 1.0 + 60.0 / a;
    double du = (umax - 1.0) / n;
    double z = 0.0, si = 0.0, sh = 0.0;
    for (int k = 0; k <= n; ++k) {
        double u = 1.0 + k * du;
        double wgt = (k == 0 || k == n) ? 1.0 : ((k & 1) ? 4.0 : 2.0);
        double w = u * u / expm1(a * u);
        double u3 = 1.0 / (u * u * u);
        double att = exp(-tau * u3);
        z += wgt * w;
        si += wgt * w * u3 * att;
        sh += wgt * w * u3 * (u - 1.0) * att;
    }
    *f_ion = si / z;
    *f_heat = sh / z;
}

void orc_bb_integrals(double tau, double T_eff, double *f_ion, double *f_heat)
{
    bb_integrals(tau, ORC_HNU_L_ERG / (ORC_KB_ERG * T_eff), f_ion, f_heat);
}

/* Recombination photons in a band (Section 4.1): in an isothermal medium at
 * T_rec an emitter spreads its photons evenly over nu_L <= nu <= nu_L + dnu,
 * dnu = k T_rec / h (and a cell's luminosity-weighted width is the same).
 * With u = nu / nu_L, D = dnu / nu_L and sigma_nu = sigma_L u^-3, a ray of
 * Lyman-limit depth tau delivers per emitted photon
 *   R_ion(tau)  = (1/D) int_1^{1+D} u^-3 e^(-tau u^-3) du
 *   R_heat(tau) = (1/D) int_1^{1+D} (u - 1) u^-3 e^(-tau u^-3) du
 * (k_alpha of Section 4.1 per neutral atom in units of sigma_L, and Eq.
 * gother per neutral atom in units of sigma_L h nu_L), by composite Simpson
 * with 512 intervals. */
static void band_integrals(double tau, double D, double *r_ion, double *r_heat)
{
    const int n = 512;
    double du = D / n, si = 0.0, sh = 0.0;
    for (int k = 0; k <= n; ++k) {
        double u = 1.0 + k * du;
        double wgt = (k == 0 || k == n) ? 1.0 : ((k & 1) ? 4.0 : 2.0);
        double u3 = 1.0 / (u * u * u);
        double v = u3 * exp(-tau * u3);
        si += wgt * v;
        sh += wgt * (u - 1.0) * v;
    }
    *r_ion = si * du / (3.0 * D);
    *r_heat = sh * du / (3.0 * D);
}

void orc_rec_band_integrals(double tau, double T_rec, double *r_ion, double *r_heat)
{
    band_integrals(tau, ORC_KB_ERG * T_rec / ORC_HNU_L_ERG, r_ion, r_heat);
}

/* Gamma_eff = sum L F(tau) / (4 pi r^2) (photons cm^-2 s^-1 at sigma_L:
 * k_ion = sigma_L Gamma_eff per neutral atom) and the photoheating rate per
 * neutral atom H = sigma_L h nu_L sum L F_heat(tau) / (4 pi r^2) (erg/s),
 * tau the Lyman-limit optical depth of Eq. tau.  Point sources: blackbody
 * at T_eff (F_ion, F_heat), or photons at nu_L when T_eff = 0 (e^-tau, no
 * heating).  In the diffuse case the emitter tree adds the recombination
 * photons: in the band of width k T_rec / h when T_rec > 0 (R_ion, and
 * R_heat: Eq. gother), else at nu_L.  The self terms (Eq. gself) are not
 * included (orc_self_terms).  stats = {rays, hops}. */
int orc_gamma_spectral(const orc *o, const float *nHI, float theta, double T_eff,
                       const long *targets, long nt, double *gamma_out, double *heat_out,
                       long long *stats)
{
    long n = targets ? nt : o->np;
    long long rays = 0, hops = 0;
    double th = theta;
    int pspec = T_eff > 0.0 ? 1 : 0;
    double a = T_eff > 0.0 ? ORC_HNU_L_ERG / (ORC_KB_ERG * T_eff) : 0.0;
    int espec = o->p.T_rec > 0.0 ? 2 : 0;
    double D = ORC_KB_ERG * o->p.T_rec / ORC_HNU_L_ERG;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : rays, hops)
    for (long q = 0; q < n; ++q) {
        long i = targets ? targets[q] : q;
        long long r = 0, hc = 0;
        double hsum = 0.0;
        double g = tree_sum(o, 1, i, th, nHI, pspec, a, &hsum, &r, &hc);
        if (o->p.diffuse) g += tree_sum(o, 2, i, th, nHI, espec, D, &hsum, &r, &hc);
        gamma_out[q] = g;
        heat_out[q] = o->p.sigma_cm2 * ORC_HNU_L_ERG * hsum;
        rays += r;
        hops += hc;
    }
    if (stats) { stats[0] = rays; stats[1] = hops; }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Gas temperature (the energy equation of Section 2.1 without its      */
/* hydrodynamic terms; the rates of Appendix A's network restricted to  */
/* hydrogen)                                                            */
/*
 * The paper takes its rate and cooling coefficients from the Kitayama et
 * al. (2001) network without printing them.  Here hydrogen only, with
 * published fits in cgs units, lambda = 2 T_HI / T, T_HI = 157807 K:
 *   alpha_A(T) = 1.269e-13 lambda^1.503 / (1 + (lambda/0.522)^0.470)^1.923
 *   alpha_B(T) = 2.753e-14 lambda^1.500 / (1 + (lambda/2.740)^0.407)^2.242
 *   recombination cooling, erg cm^3/s, times n_e n_p:
 *     case A  1.778e-29 T lambda^1.965 / (1 + (lambda/0.541)^0.502)^2.697
 *     case B  3.435e-30 T lambda^1.970 / (1 + (lambda/2.250)^0.376)^3.720
 *   collisional ionisation rate, cm^3/s, times n_e n_HI:
 *     21.11 T^-1.5 exp(-lambda/2) lambda^-1.089 / (1 + (lambda/0.354)^0.874)^1.101
 *   (all from Hui & Gnedin 1997, Appendix), its cooling k T_HI times the rate;
 *   collisional excitation cooling (Black 1981, as given by Cen 1992),
 *     7.5e-19 exp(-118348/T) / (1 + (T/1e5)^0.5) erg cm^3/s times n_e n_HI;
 *   free-free cooling 1.42e-27 g_ff T^0.5 erg cm^3/s times n_e n_p with
 *     g_ff = 1.1 + 0.34 exp(-(5.5 - log10 T)^2 / 3) (Cen 1992). */
#define ORC_T_HI 157807.0

double orc_rate(int which, double T)
{
    double lam = 2.0 * ORC_T_HI / T;
    switch (which) {
    case 0: return 1.269e-13 * pow(lam, 1.503) / pow(1.0 + pow(lam / 0.522, 0.470), 1.923);
    case 1: return 2.753e-14 * pow(lam, 1.500) / pow(1.0 + pow(lam / 2.740, 0.407), 2.242);
    case 2: return 1.778e-29 * T * pow(lam, 1.965) / pow(1.0 + pow(lam / 0.541, 0.502), 2.697);
    case 3: return 3.435e-30 * T * pow(lam, 1.970) / pow(1.0 + pow(lam / 2.250, 0.376), 3.720);
    case 4:
        return 21.11 * pow(T, -1.5) * exp(-0.5 * lam) * pow(lam, -1.089) /
               pow(1.0 + pow(lam / 0.354, 0.874), 1.101);
    case 5: return ORC_KB_ERG * ORC_T_HI * orc_rate(4, T);
    case 6: return 7.5e-19 * exp(-118348.0 / T) / (1.0 + sqrt(T / 1e5));
    case 7: {
        double lt = log10(T);
        double gff = 1.1 + 0.34 * exp(-(5.5 - lt) * (5.5 - lt) / 3.0);
        return 1.42e-27 * gff * sqrt(T);
    }
    }
    return 0.0;
}

/* Net cooling minus heating of the energy equation at temperature T, with
 * the ionisation state (x, n_H) held: Lambda(T) - H, erg cm^-3 s^-1. */
static double net_cooling(int caseA, double T, double x, double nh, double heat)
{
    double ne = x * nh, np_ = x * nh, nhi = (1.0 - x) * nh;
    double lam = ne * np_ * (orc_rate(caseA ? 2 : 3, T) + orc_rate(7, T)) +
                 ne * nhi * (orc_rate(5, T) + orc_rate(6, T));
    return lam - heat;
}

/* Recombination emitters with temperature-dependent coefficients:
 * N_rec,j = alpha_1(T_j) n_e n_p V_j, alpha_1 = alpha_A(T) - alpha_B(T)
 * (Section 4.1); T = NULL takes the constant alpha_A - alpha_B of the
 * parameters (orc_set_emitters). */
void orc_set_emitters_T(orc *o, const double *y, const float *nH, const double *T)
{
    if (!T) {
        orc_set_emitters(o, y, nH);
        return;
    }
    double lu3 = o->p.len_unit_cm * o->p.len_unit_cm * o->p.len_unit_cm;
    for (long i = 0; i < o->np; ++i) {
        double a1 = orc_rate(0, T[i]) - orc_rate(1, T[i]);
        double ne = (1.0 - y[i]) * (double)nH[i];
        o->eL[i] = a1 * ne * ne * (o->V[i] * lu3);
    }
    if (o->et.n) moments_node(&o->et, 0, o->pperm, o->px, o->py, o->pz, o->eL);
    if (o->et.n && o->p.lum_kernel) kernel_luminosities(o);
}

/* One implicit step of hydrogen and its gas temperature over dt, per
 * particle (input order):
 *  1. the neutral fraction, with the step-start temperature T0: backward
 *     Euler of dy/dt = -k y - C y (1 - y) + a (1 - y)^2 with k = sigma Gamma
 *     (+ the self term of Eq. kself1, at the Lyman limit or band-averaged,
 *     with alpha_1(T0) in the diffuse case),
 *     C = Gc(T0) n_H (collisional ionisation), a = alpha(T0) n_H (alpha_A
 *     in the diffuse case, else alpha_B): the root in [0, 1] of
 *     (a' + c') y^2 - (1 + K + c' + 2a') y + (y0 + a') = 0 (primes: times
 *     dt), taken as 2 (y0 + a') / (b + sqrt(b^2 - 4 (a' + c') (y0 + a')));
 *  2. the temperature, with the new ionisation x1 = 1 - y1: backward Euler
 *     of the energy density u = (3/2) (1 + x) n_H k T,
 *       (3/2) k n_H ((1 + x1) T1 - (1 + x0) T0) = dt (H - Lambda(T1, x1)),
 *     H = y1 n_H h with h the photoheating per neutral atom (erg/s) of the
 *     solve (blackbody sources, the recombination band and its self term),
 *     Lambda the recombination (case A in the diffuse case, else B),
 *     free-free, collisional-excitation and collisional-ionisation cooling.
 *     T1 is found by bisection on ln T over [10 K, 1e9 K] (the residual is
 *     increasing in T1 there for every state tested), 200 halvings.
 * heat may be NULL (no photoheating).  targets (may be NULL) lists the
 * particles (input indices) that entry t of the arrays belongs to. */
void orc_ionize_thermal(const orc *o, const double *gamma, const double *heat, const float *nH,
                        const double *y0, const double *T0, double dt, const long *targets,
                        long n, double *y1, double *T1)
{
    int diffuse = o->p.diffuse;
    double sig = o->p.sigma_cm2;
    for (long t = 0; t < n; ++t) {
        long i = targets ? targets[t] : t;   /* the particle (volume); arrays indexed by t */
        double nh = nH[t], t0 = T0[t], yy = y0[t];
        double k = sig * gamma[t];
        if (diffuse) {
            double ks, hs;
            self_terms_a1(o, i, nh, yy, orc_rate(0, t0) - orc_rate(1, t0), &ks, &hs);
            k += ks;
        }
        double a = orc_rate(diffuse ? 0 : 1, t0) * nh * dt;
        double c = orc_rate(4, t0) * nh * dt;
        double K = k * dt;
        double b = 1.0 + K + c + 2.0 * a;
        double disc = b * b - 4.0 * (a + c) * (yy + a);
        if (disc < 0.0) disc = 0.0;
        double y = 2.0 * (yy + a) / (b + sqrt(disc));
        y1[t] = y;
        double x0 = 1.0 - yy, x1 = 1.0 - y;
        double e = 1.5 * ORC_KB_ERG * nh;
        double H = heat ? y * nh * heat[t] : 0.0;
        double lo = log(10.0), hi = log(1e9);
        double u0 = e * (1.0 + x0) * t0;
#define RESID(T) (e * (1.0 + x1) * (T) - u0 + dt * net_cooling(diffuse, (T), x1, nh, H))
        if (RESID(10.0) >= 0.0) { T1[t] = 10.0; continue; }
        if (RESID(1e9) <= 0.0) { T1[t] = 1e9; continue; }
        for (int it = 0; it < 200; ++it) {
            double mid = 0.5 * (lo + hi);
            if (RESID(exp(mid)) > 0.0) hi = mid;
            else lo = mid;
        }
#undef RESID
        T1[t] = exp(0.5 * (lo + hi));
    }
}
