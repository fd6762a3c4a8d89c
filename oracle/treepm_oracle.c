/*
 * treepm_oracle.c -- plain, slow CPU FP64 oracle of the short-range TreePM path
 * of Ishiyama, Nitadori & Makino (SC12, "4.45 Pflops astrophysical N-body
 * simulation on K computer").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code with the CUDA library.
 *
 * Everything is FP64, round-to-nearest, compiled with -ffp-contract=off so that
 * every multiply and add rounds separately.  The pieces, in the order the
 * method runs them:
 *
 *   or_g, or_gpx        cutoff function g_P3M of Eq. 3 and its derivative g'/xi
 *   pair_acc            one term of the particle-particle sum of Eq. 2, with
 *                       Plummer softening on the 1/r^3 factor (Sec. II) and
 *                       minimum-image periodic distance (Sec. I)
 *   or_brute_force      Eq. 2 summed over all j != i (plain definition)
 *   or_build            Morton keys, sort, octree (Sec. I, tree algorithm),
 *                       node monopoles, particle groups (Sec. II, Barnes'
 *                       modified algorithm)
 *   or_lists            per-group interaction lists: cut at r_cut, monopole
 *                       opening criterion theta (Sec. I and II)
 *   or_list_forces      Eq. 2 over each group's list (nodes as monopoles)
 *   or_list_vjp         the vector-Jacobian product of or_list_forces
 *   or_count_useful     how many evaluated pairs lie inside the cutoff
 *
 * Readings where the paper is silent (every one is listed in the design notes):
 *   - softening: 1/|r|^3 -> 1/(r^2+eps^2)^{3/2}; the cutoff argument uses the
 *     unsoftened r; pairs with r >= r_cut or r == 0 contribute exactly 0.
 *     Every force and adjoint function also takes xi_soft, a bitmask: bit 1
 *     selects the softened cutoff argument below, bit 2 the paper's refined
 *     inverse square root (or_rsqrt_refined) for 1/s^3.  With bit 1 set, the
 *     cutoff argument is the softened distance s = sqrt(r^2 + eps^2) instead
 *     (the paper's kernel form), and pairs with s >= r_cut contribute 0.
 *   - keys: x wrapped to [0,1), quantised to 21 bits, x bit highest in each
 *     interleaved triplet; ties in the sort broken by input index.
 *   - octree: a node splits while count > n_leaf and level < 21; children in
 *     octant order; empty children omitted; nodes numbered breadth first.
 *   - monopole: mass and centre of mass summed sequentially in particle order
 *     (leaves) or octant order (internal nodes).
 *   - groups: under each node holding more than n_crit particles, each maximal
 *     run of consecutive children (octant order) holding <= n_crit particles
 *     is cut into balanced groups of at most n_crit particles; a leaf holding
 *     more than n_crit particles is a group by itself.
 *   - lists: prune when the periodic box-to-box gap d is >= r_cut; accept a
 *     node as a monopole (at its centre of mass) when it does not overlap the
 *     group, lies entirely inside r_cut of every point of the group box (largest
 *     box-to-box distance < r_cut, so that no monopole straddles the cutoff
 *     sphere) and (l/d)^2 < theta^2 with l = 2^-level; otherwise open it; at an
 *     opened leaf keep particles whose point-to-box gap is < r_cut.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAX_LEVEL 21
#define OR_QSCALE 2097152.0 /* 2^21 */

/* ------------------------------------------------------------------------ */
/* Eq. 3: the cutoff shape g_P3M(xi), exactly as printed (nested form plus   */
/* the zeta^6 correction, zeta = max(0, xi - 1)); zero for xi > 2.           */
/* ------------------------------------------------------------------------ */
double or_g(double xi)
{
    if (xi > 2.0) return 0.0;
    double zeta = xi - 1.0;
    if (zeta < 0.0) zeta = 0.0;
    double inner = -8.0 / 5.0 +
                   xi * xi * (8.0 / 5.0 + xi * (-1.0 / 2.0 + xi * (-12.0 / 35.0 + xi * (3.0 / 20.0))));
    double z2 = zeta * zeta;
    double z6 = z2 * z2 * z2;
    return 1.0 + xi * xi * xi * inner - z6 * (3.0 / 35.0 + xi * (18.0 / 35.0 + xi * (1.0 / 5.0)));
}

/* g'(xi)/xi: Eq. 3 differentiated term by term.  With g = 1 + xi^3 P(xi) -
 * zeta^6 Q(xi), P = -8/5 + 8/5 xi^2 - 1/2 xi^3 - 12/35 xi^4 + 3/20 xi^5 and
 * Q = 3/35 + 18/35 xi + 1/5 xi^2:
 *   g'/xi = 3 xi P + xi^2 P' - (6 zeta^5 Q + zeta^6 Q') / xi.               */
double or_gpx(double xi)
{
    if (xi > 2.0) return 0.0;
    double P = -8.0 / 5.0 + xi * xi * (8.0 / 5.0 + xi * (-1.0 / 2.0 + xi * (-12.0 / 35.0 + xi * (3.0 / 20.0))));
    double Pp = xi * (16.0 / 5.0 + xi * (-3.0 / 2.0 + xi * (-48.0 / 35.0 + xi * (3.0 / 4.0))));
    double r = 3.0 * xi * P + xi * xi * Pp;
    double zeta = xi - 1.0;
    if (zeta > 0.0) {
        double Q = 3.0 / 35.0 + xi * (18.0 / 35.0 + xi * (1.0 / 5.0));
        double Qp = 18.0 / 35.0 + xi * (2.0 / 5.0);
        double z5 = zeta * zeta * zeta * zeta * zeta;
        r -= (6.0 * z5 * Q + z5 * zeta * Qp) / xi;
    }
    return r;
}

/* Periodic minimum image of a coordinate difference (unit box, Sec. I). */
static inline double minimg(double t) { return t - rint(t); }

typedef struct {
    double G, eps, rcut, theta;
    double rc2, eps2, th2;
    int soft;                  /* cutoff argument from the softened distance */
    int rsq;                   /* 1/s from the refined estimate (or_rsqrt_refined) */
} or_prm;

/* The paper's inverse square root (Sec. II-A): a low-accuracy estimate y0 of
 * 1/sqrt(x) refined by one third-order step, h0 = 1 - x y0^2 and
 * y1 = y0 (1 + h0/2 + 3 h0^2/8).  With y0 = (1 + e)/sqrt(x) the result is
 * (1 + 5/2 e^3 + 15/8 e^4 + 3/8 e^5)/sqrt(x) exactly.                     */
double or_rsqrt_third_order(double x, double y0)
{
    double h0 = 1.0 - x * (y0 * y0);
    return y0 * ((1.0 + 0.5 * h0) + 0.375 * (h0 * h0));
}

/* The estimate the refinement starts from.  The K computer's instruction gives
 * 8 bits; a GPU has no such instruction, and its counterpart here is the
 * integer estimate of Lomont (2003, "Fast inverse square root"): the FP32 bit
 * pattern of x shifted right by one and subtracted from 0x5f3759df (relative
 * error below 3.5e-2), improved by one Newton step y (3/2 - x y^2/2) to below
 * 1.8e-3, about the paper's 8 to 9 bits.  x > 0 and finite.                 */
double or_rsqrt_seed(double x)
{
    float xf = (float)x, yf;
    uint32_t b;
    memcpy(&b, &xf, sizeof b);
    b = 0x5f3759dfu - (b >> 1);
    memcpy(&yf, &b, sizeof yf);
    double y = (double)yf;
    return y * (1.5 - (0.5 * x) * (y * y));
}

/* 1/sqrt(x) by the paper's refinement of the estimate above: relative error
 * 5/2 e^3 + O(e^4) <= 1.5e-8 for |e| <= 1.8e-3.                            */
double or_rsqrt_refined(double x)
{
    return or_rsqrt_third_order(x, or_rsqrt_seed(x));
}

static or_prm make_prm(double G, double eps, double rcut, double theta)
{
    or_prm p;
    p.G = G; p.eps = eps; p.rcut = rcut; p.theta = theta;
    p.rc2 = rcut * rcut; p.eps2 = eps * eps; p.th2 = theta * theta;
    p.soft = 0;
    p.rsq = 0;
    return p;
}

/* variant: bit 1 = softened cutoff argument, bit 2 = refined inverse square
 * root (the "xi_soft" argument of the functions below). */
static or_prm make_prm_xi(double G, double eps, double rcut, int xi_soft)
{
    or_prm p = make_prm(G, eps, rcut, 0.0);
    p.soft = (xi_soft & 1) != 0;
    p.rsq = (xi_soft & 2) != 0;
    return p;
}

/* 1/s^3 and 1/s^2 from s^2: exact, or through the paper's refinement. */
static inline void inv_s3(const or_prm *P, double s2, double *is3, double *is2)
{
    if (P->rsq) {
        double y = or_rsqrt_refined(s2);
        *is2 = y * y;
        *is3 = *is2 * y;
    } else {
        *is3 = 1.0 / (s2 * sqrt(s2));
        *is2 = 1.0 / s2;
    }
}

/* One term of Eq. 2: acceleration of i due to mass mj at minimum-image offset
 * d = x_j - x_i, softened on the 1/r^3 factor, cut by g(2c/r_cut).  The cutoff
 * argument c is the plain distance r by default; in the softened-xi variant it
 * is s = sqrt(r^2 + eps^2), the distance the paper's kernel takes from its one
 * inverse square root per pair (Sec. II-A), so the term vanishes for s >= r_cut. */
static inline void pair_acc(double dx, double dy, double dz, double mj,
                            const or_prm *P, double *ax, double *ay, double *az)
{
    double r2 = (dx * dx + dy * dy) + dz * dz;
    if (r2 == 0.0) return;
    double s2 = r2 + P->eps2;
    double c2 = P->soft ? s2 : r2;
    if (!(c2 < P->rc2)) return;
    double g = or_g(2.0 * sqrt(c2) / P->rcut);
    double fac;
    if (P->rsq) {
        double is3, is2;
        inv_s3(P, s2, &is3, &is2);
        fac = P->G * mj * g * is3;
    } else {
        fac = P->G * mj * g / (s2 * sqrt(s2));
    }
    *ax += fac * dx;
    *ay += fac * dy;
    *az += fac * dz;
}

/* v = G mj J(d) w with J = phi I + (phi'/r) d d^T the Jacobian of
 * d * phi(|d|), phi = g(xi)/s^3:  phi'/r = (2/r_cut)^2 (g'/xi)/s^3 - 3 g/s^5.
 * The same expression holds in the softened-xi variant (xi = 2s/r_cut): there
 * dphi/dd = (g'(xi) (2/r_cut)/s^4 - 3 g/s^5) d, and (2/r_cut)/s^4 equals
 * (2/r_cut)^2/(xi s^3). */
static inline void pair_jw(double dx, double dy, double dz, double mj,
                           const double *w, const or_prm *P, double *v)
{
    v[0] = v[1] = v[2] = 0.0;
    double r2 = (dx * dx + dy * dy) + dz * dz;
    if (r2 == 0.0) return;
    double s2 = r2 + P->eps2;
    double c2 = P->soft ? s2 : r2;
    if (!(c2 < P->rc2)) return;
    double xi = 2.0 * sqrt(c2) / P->rcut;
    double g = or_g(xi);
    double gp = or_gpx(xi);
    double k = 2.0 / P->rcut;
    double phi, dphi;
    if (P->rsq) {
        double is3, is2;
        inv_s3(P, s2, &is3, &is2);
        phi = g * is3;
        dphi = k * k * gp * is3 - 3.0 * g * (is3 * is2);
    } else {
        double s3 = s2 * sqrt(s2);
        phi = g / s3;
        dphi = k * k * gp / s3 - 3.0 * g / (s3 * s2);
    }
    double dw = (dx * w[0] + dy * w[1]) + dz * w[2];
    double c = P->G * mj;
    v[0] = c * (phi * w[0] + dphi * dw * dx);
    v[1] = c * (phi * w[1] + dphi * dw * dy);
    v[2] = c * (phi * w[2] + dphi * dw * dz);
}

/* Public single-pair helpers (tests pin these against closed forms). */
void or_pair(const double *d, double mj, double G, double eps, double rcut, double *acc,
             int xi_soft)
{
    or_prm P = make_prm_xi(G, eps, rcut, xi_soft);
    acc[0] = acc[1] = acc[2] = 0.0;
    pair_acc(minimg(d[0]), minimg(d[1]), minimg(d[2]), mj, &P, &acc[0], &acc[1], &acc[2]);
}

void or_pair_jw(const double *d, double mj, const double *w, double G, double eps,
                double rcut, double *v, int xi_soft)
{
    or_prm P = make_prm_xi(G, eps, rcut, xi_soft);
    pair_jw(minimg(d[0]), minimg(d[1]), minimg(d[2]), mj, w, &P, v);
}

/* Wrap into the unit box: x - floor(x), with the rounding case 1.0 -> 0.0. */
static inline double wrap01(double x)
{
    double w = x - floor(x);
    if (w >= 1.0) w = 0.0;
    return w;
}

/* ------------------------------------------------------------------------ */
/* Eq. 2 summed directly over every other particle (the plain definition).  */
/* ------------------------------------------------------------------------ */
void or_brute_force(int64_t n, const double *pos, const double *mass, double G,
                    double eps, double rcut, double *acc, int xi_soft)
{
    or_prm P = make_prm_xi(G, eps, rcut, xi_soft);
    double *w = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < 3 * n; i++) w[i] = wrap01(pos[i]);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++) {
        double ax = 0, ay = 0, az = 0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            pair_acc(minimg(w[3 * j] - w[3 * i]), minimg(w[3 * j + 1] - w[3 * i + 1]),
                     minimg(w[3 * j + 2] - w[3 * i + 2]), mass[j], &P, &ax, &ay, &az);
        }
        acc[3 * i] = ax; acc[3 * i + 1] = ay; acc[3 * i + 2] = az;
    }
    free(w);
}

/* The same sum for a sample of targets idx[0..ns) only (large boxes). */
void or_brute_force_sample(int64_t n, const double *pos, const double *mass, double G,
                           double eps, double rcut, int64_t ns, const int64_t *idx,
                           double *acc, int xi_soft)
{
    or_prm P = make_prm_xi(G, eps, rcut, xi_soft);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t s = 0; s < ns; s++) {
        int64_t i = idx[s];
        double xi = wrap01(pos[3 * i]), yi = wrap01(pos[3 * i + 1]), zi = wrap01(pos[3 * i + 2]);
        double ax = 0, ay = 0, az = 0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            pair_acc(minimg(wrap01(pos[3 * j]) - xi), minimg(wrap01(pos[3 * j + 1]) - yi),
                     minimg(wrap01(pos[3 * j + 2]) - zi), mass[j], &P, &ax, &ay, &az);
        }
        acc[3 * s] = ax; acc[3 * s + 1] = ay; acc[3 * s + 2] = az;
    }
}

/* Gradient of L = sum_i w_i . a_i for the direct sum:
 * dL/dx_k = G sum_{j != k} J(x_j - x_k) (m_k w_j - m_j w_k). */
void or_brute_vjp(int64_t n, const double *pos, const double *mass, double G, double eps,
                  double rcut, const double *wv, double *grad, int xi_soft)
{
    or_prm P = make_prm_xi(G, eps, rcut, xi_soft);
    double *x = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < 3 * n; i++) x[i] = wrap01(pos[i]);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < n; k++) {
        double gk[3] = {0, 0, 0};
        for (int64_t j = 0; j < n; j++) {
            if (j == k) continue;
            double u[3];
            for (int c = 0; c < 3; c++) u[c] = mass[k] * wv[3 * j + c] - mass[j] * wv[3 * k + c];
            double v[3];
            /* J(d) u with unit mass and G folded in below */
            pair_jw(minimg(x[3 * j] - x[3 * k]), minimg(x[3 * j + 1] - x[3 * k + 1]),
                    minimg(x[3 * j + 2] - x[3 * k + 2]), 1.0, u, &P, v);
            gk[0] += v[0]; gk[1] += v[1]; gk[2] += v[2];
        }
        grad[3 * k] = gk[0]; grad[3 * k + 1] = gk[1]; grad[3 * k + 2] = gk[2];
    }
    free(x);
}

/* The same gradient for a sample of particles idx[0..ns) only (large boxes):
 * row s of the result is dL/dx_{idx[s]}. */
void or_brute_vjp_sample(int64_t n, const double *pos, const double *mass, double G, double eps,
                         double rcut, const double *wv, int64_t ns, const int64_t *idx, double *grad,
                         int xi_soft)
{
    or_prm P = make_prm_xi(G, eps, rcut, xi_soft);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t s = 0; s < ns; s++) {
        int64_t k = idx[s];
        double xk = wrap01(pos[3 * k]), yk = wrap01(pos[3 * k + 1]), zk = wrap01(pos[3 * k + 2]);
        double gk[3] = {0, 0, 0};
        for (int64_t j = 0; j < n; j++) {
            if (j == k) continue;
            double u[3], v[3];
            for (int c = 0; c < 3; c++) u[c] = mass[k] * wv[3 * j + c] - mass[j] * wv[3 * k + c];
            pair_jw(minimg(wrap01(pos[3 * j]) - xk), minimg(wrap01(pos[3 * j + 1]) - yk),
                    minimg(wrap01(pos[3 * j + 2]) - zk), 1.0, u, &P, v);
            gk[0] += v[0]; gk[1] += v[1]; gk[2] += v[2];
        }
        grad[3 * s] = gk[0]; grad[3 * s + 1] = gk[1]; grad[3 * s + 2] = gk[2];
    }
}

/* ------------------------------------------------------------------------ */
/* Morton keys (tree algorithm, Sec. I): 21 bits per axis, x bit highest.    */
/* ------------------------------------------------------------------------ */
uint64_t or_morton(uint32_t qx, uint32_t qy, uint32_t qz)
{
    uint64_t key = 0;
    for (int b = 0; b < OR_MAX_LEVEL; b++) {
        key |= (uint64_t)((qx >> b) & 1u) << (3 * b + 2);
        key |= (uint64_t)((qy >> b) & 1u) << (3 * b + 1);
        key |= (uint64_t)((qz >> b) & 1u) << (3 * b);
    }
    return key;
}

static inline uint32_t quantise(double w)
{
    double q = floor(w * OR_QSCALE);
    if (q > OR_QSCALE - 1.0) q = OR_QSCALE - 1.0;
    if (q < 0.0) q = 0.0;
    return (uint32_t)q;
}

uint64_t or_key_of(double x, double y, double z)
{
    return or_morton(quantise(wrap01(x)), quantise(wrap01(y)), quantise(wrap01(z)));
}

/* ------------------------------------------------------------------------ */
/* Tree                                                                     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n;
    int32_t n_leaf, n_crit;
    /* particles in key order */
    uint64_t *key;
    int64_t *perm;            /* perm[s] = input index of sorted particle s */
    double *x[3], *m;         /* wrapped positions, masses (sorted)         */
    double *xb[3];            /* positions the moments were last taken from */
    /* nodes, breadth-first numbering */
    int64_t n_nodes, cap_nodes;
    int32_t *level;
    int64_t *first, *count, *child, *nchild, *parent;
    double *M, *S[3], *com[3], *lo[3], *hi[3], *cen[3], *half[3];
    /* groups */
    int64_t n_groups, cap_groups;
    int64_t *gfirst, *gcount;
    double *gc[3], *gh[3];
    /* lists */
    int64_t *loff;            /* [n_groups+1] */
    int64_t n_entries;
    int64_t *ent;             /* >= 0 sorted particle, < 0 node -(id+1)     */
} or_tree;

typedef struct { uint64_t key; int64_t idx; } kv_t;

static int kv_cmp(const void *a, const void *b)
{
    const kv_t *p = (const kv_t *)a, *q = (const kv_t *)b;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    if (p->idx != q->idx) return p->idx < q->idx ? -1 : 1;
    return 0;
}

static void node_reserve(or_tree *t, int64_t need)
{
    if (need <= t->cap_nodes) return;
    int64_t cap = t->cap_nodes ? t->cap_nodes : 64;
    while (cap < need) cap *= 2;
#define RE(p, T) p = (T *)realloc(p, sizeof(T) * (size_t)cap)
    RE(t->level, int32_t); RE(t->first, int64_t); RE(t->count, int64_t);
    RE(t->child, int64_t); RE(t->nchild, int64_t); RE(t->parent, int64_t);
    RE(t->M, double);
    for (int c = 0; c < 3; c++) {
        RE(t->S[c], double); RE(t->com[c], double); RE(t->lo[c], double);
        RE(t->hi[c], double); RE(t->cen[c], double); RE(t->half[c], double);
    }
#undef RE
    t->cap_nodes = cap;
}

static int64_t node_push(or_tree *t, int32_t level, int64_t first, int64_t count, int64_t parent)
{
    node_reserve(t, t->n_nodes + 1);
    int64_t id = t->n_nodes++;
    t->level[id] = level; t->first[id] = first; t->count[id] = count;
    t->parent[id] = parent; t->child[id] = -1; t->nchild[id] = 0;
    return id;
}

static int is_leaf(const or_tree *t, int64_t i) { return t->nchild[i] == 0; }

/* Monopoles bottom-up in canonical order: a leaf sums its particles in key
 * order, an internal node sums its children in octant order; every multiply
 * and add rounds separately.  COM = S / M.  When `boxes` is set the tight
 * bounding box (min/max of member positions) and its centre/half-width
 * (lo+hi)*0.5, (hi-lo)*0.5 are recomputed too. */
static void moments(or_tree *t, int boxes)
{
    for (int64_t i = t->n_nodes - 1; i >= 0; i--) {
        double M = 0.0, S[3] = {0.0, 0.0, 0.0}, lo[3], hi[3];
        for (int c = 0; c < 3; c++) { lo[c] = INFINITY; hi[c] = -INFINITY; }
        if (is_leaf(t, i)) {
            for (int64_t p = t->first[i]; p < t->first[i] + t->count[i]; p++) {
                M = M + t->m[p];
                for (int c = 0; c < 3; c++) {
                    double mx = t->m[p] * t->xb[c][p];
                    S[c] = S[c] + mx;
                    if (t->xb[c][p] < lo[c]) lo[c] = t->xb[c][p];
                    if (t->xb[c][p] > hi[c]) hi[c] = t->xb[c][p];
                }
            }
        } else {
            for (int64_t k = t->child[i]; k < t->child[i] + t->nchild[i]; k++) {
                M = M + t->M[k];
                for (int c = 0; c < 3; c++) {
                    S[c] = S[c] + t->S[c][k];
                    if (t->lo[c][k] < lo[c]) lo[c] = t->lo[c][k];
                    if (t->hi[c][k] > hi[c]) hi[c] = t->hi[c][k];
                }
            }
        }
        t->M[i] = M;
        for (int c = 0; c < 3; c++) {
            t->S[c][i] = S[c];
            if (boxes) {
                t->lo[c][i] = lo[c];
                t->hi[c][i] = hi[c];
                t->cen[c][i] = (lo[c] + hi[c]) * 0.5;
                t->half[c][i] = (hi[c] - lo[c]) * 0.5;
            }
            t->com[c][i] = M > 0.0 ? S[c] / M : t->cen[c][i];
        }
    }
}

static void group_push(or_tree *t, int64_t first, int64_t count)
{
    if (t->n_groups == t->cap_groups) {
        int64_t cap = t->cap_groups ? 2 * t->cap_groups : 64;
        t->gfirst = (int64_t *)realloc(t->gfirst, sizeof(int64_t) * (size_t)cap);
        t->gcount = (int64_t *)realloc(t->gcount, sizeof(int64_t) * (size_t)cap);
        t->cap_groups = cap;
    }
    t->gfirst[t->n_groups] = first;
    t->gcount[t->n_groups] = count;
    t->n_groups++;
}

/* A run of consecutive small siblings holding S particles is cut into
 * kg = ceil(S / n_crit) groups of about ceil(S / kg): siblings are added in
 * octant order and a group is closed before a sibling that would push it past
 * n_crit, or once it has reached that target size. */
static void flush_run(or_tree *t, const int64_t *run, int k)
{
    if (k == 0) return;
    int64_t S = 0;
    for (int a = 0; a < k; a++) S += t->count[run[a]];
    int64_t nc = t->n_crit;
    int64_t kg = (S + nc - 1) / nc;
    int64_t target = (S + kg - 1) / kg;
    int64_t cur = 0, cur_first = -1;
    for (int a = 0; a < k; a++) {
        int64_t c = t->count[run[a]];
        if (cur > 0 && (cur + c > nc || cur >= target)) {
            group_push(t, cur_first, cur);
            cur = 0;
        }
        if (cur == 0) cur_first = t->first[run[a]];
        cur += c;
    }
    if (cur > 0) group_push(t, cur_first, cur);
}

/* Visit a node holding more than n_crit particles that has children. */
static void group_visit(or_tree *t, int64_t i)
{
    int64_t run[8];
    int k = 0;
    for (int64_t c = t->child[i]; c < t->child[i] + t->nchild[i]; c++) {
        if (t->count[c] > t->n_crit) {
            flush_run(t, run, k);
            k = 0;
            if (is_leaf(t, c)) group_push(t, t->first[c], t->count[c]);
            else group_visit(t, c);
        } else {
            run[k++] = c;
        }
    }
    flush_run(t, run, k);
}

void or_free(or_tree *t);

/* Build keys, sort, octree, monopoles and groups for one periodic unit box.
 * mass == NULL means equal masses 1/n.  Returns NULL on bad arguments. */
or_tree *or_build(int64_t n, const double *pos, const double *mass, int32_t n_leaf,
                  int32_t n_crit)
{
    if (n < 0 || n_leaf < 1 || n_crit < 1) return NULL;
    or_tree *t = (or_tree *)calloc(1, sizeof(or_tree));
    t->n = n; t->n_leaf = n_leaf; t->n_crit = n_crit;
    size_t nn = (size_t)(n > 0 ? n : 1);
    t->key = (uint64_t *)malloc(sizeof(uint64_t) * nn);
    t->perm = (int64_t *)malloc(sizeof(int64_t) * nn);
    t->m = (double *)malloc(sizeof(double) * nn);
    for (int c = 0; c < 3; c++) {
        t->x[c] = (double *)malloc(sizeof(double) * nn);
        t->xb[c] = (double *)malloc(sizeof(double) * nn);
    }
    kv_t *kv = (kv_t *)malloc(sizeof(kv_t) * nn);
    for (int64_t i = 0; i < n; i++) {
        kv[i].key = or_key_of(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]);
        kv[i].idx = i;
    }
    qsort(kv, (size_t)n, sizeof(kv_t), kv_cmp);
    for (int64_t s = 0; s < n; s++) {
        int64_t i = kv[s].idx;
        t->key[s] = kv[s].key;
        t->perm[s] = i;
        t->m[s] = mass ? mass[i] : 1.0 / (double)n;
        for (int c = 0; c < 3; c++) {
            t->x[c][s] = wrap01(pos[3 * i + c]);
            t->xb[c][s] = t->x[c][s];
        }
    }
    free(kv);
    if (n == 0) return t;

    /* breadth-first octree: node ids are assigned in queue order */
    node_push(t, 0, 0, n, -1);
    for (int64_t i = 0; i < t->n_nodes; i++) {
        if (t->count[i] <= n_leaf || t->level[i] >= OR_MAX_LEVEL) continue;
        int shift = 3 * (OR_MAX_LEVEL - 1 - t->level[i]);
        int64_t p = t->first[i], end = t->first[i] + t->count[i];
        int64_t first_child = t->n_nodes, nc = 0;
        for (uint64_t o = 0; o < 8; o++) {
            int64_t q = p;
            while (q < end && ((t->key[q] >> shift) & 7u) == o) q++;
            if (q > p) {
                node_push(t, t->level[i] + 1, p, q - p, i);
                nc++;
            }
            p = q;
        }
        t->child[i] = first_child;
        t->nchild[i] = nc;
    }
    moments(t, 1);

    /* groups */
    if (t->count[0] <= n_crit || is_leaf(t, 0)) group_push(t, 0, n);
    else group_visit(t, 0);
    for (int c = 0; c < 3; c++) {
        t->gc[c] = (double *)malloc(sizeof(double) * (size_t)t->n_groups);
        t->gh[c] = (double *)malloc(sizeof(double) * (size_t)t->n_groups);
    }
    for (int64_t g = 0; g < t->n_groups; g++) {
        for (int c = 0; c < 3; c++) {
            double lo = INFINITY, hi = -INFINITY;
            for (int64_t p = t->gfirst[g]; p < t->gfirst[g] + t->gcount[g]; p++) {
                if (t->x[c][p] < lo) lo = t->x[c][p];
                if (t->x[c][p] > hi) hi = t->x[c][p];
            }
            t->gc[c][g] = (lo + hi) * 0.5;
            t->gh[c][g] = (hi - lo) * 0.5;
        }
    }
    return t;
}

/* ------------------------------------------------------------------------ */
/* Interaction lists (Barnes' modified algorithm, Sec. II; cutoff, Sec. II)   */
/* ------------------------------------------------------------------------ */
/* Periodic box-to-box distances between the box (a, h) and the group box
 * (c, hg).  Per axis t = minimg(a - c), s = h + hg, gap = max(0, |t| - s),
 * far = |t| + s; returns gap2 = (gx*gx + gy*gy) + gz*gz and far2 likewise. */
static inline double box_dist2(const double *a, const double *h, const double *c,
                               const double *hg, double *far2)
{
    double g[3], f[3];
    for (int k = 0; k < 3; k++) {
        double tt = fabs(minimg(a[k] - c[k]));
        double s = h[k] + hg[k];
        double e = tt - s;
        g[k] = e > 0.0 ? e : 0.0;
        f[k] = tt + s;
    }
    if (far2) *far2 = (f[0] * f[0] + f[1] * f[1]) + f[2] * f[2];
    return (g[0] * g[0] + g[1] * g[1]) + g[2] * g[2];
}

typedef struct { int64_t *v; int64_t n, cap; } ivec;

static inline void ivec_push(ivec *a, int64_t x)
{
    if (a->n == a->cap) {
        a->cap = a->cap ? 2 * a->cap : 256;
        a->v = (int64_t *)realloc(a->v, sizeof(int64_t) * (size_t)a->cap);
    }
    a->v[a->n++] = x;
}

static void walk(const or_tree *t, int64_t i, int64_t g, const or_prm *P, ivec *out)
{
    double cg[3], hg[3], cn[3], hn[3], zero[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < 3; k++) {
        cg[k] = t->gc[k][g]; hg[k] = t->gh[k][g];
        cn[k] = t->cen[k][i]; hn[k] = t->half[k][i];
    }
    double far2;
    double gap2 = box_dist2(cn, hn, cg, hg, &far2);
    if (gap2 >= P->rc2) return;                                      /* prune */
    int64_t g0 = t->gfirst[g], g1 = g0 + t->gcount[g];
    int64_t n0 = t->first[i], n1 = n0 + t->count[i];
    int overlap = n0 < g1 && g0 < n1;
    double l = ldexp(1.0, -t->level[i]);
    if (!overlap && far2 < P->rc2 && l * l < P->th2 * gap2) {        /* accept */
        ivec_push(out, -(i + 1));
        return;
    }
    if (is_leaf(t, i)) {
        for (int64_t p = n0; p < n1; p++) {
            double xp[3] = {t->x[0][p], t->x[1][p], t->x[2][p]};
            if (box_dist2(xp, zero, cg, hg, NULL) < P->rc2) ivec_push(out, p);
        }
        return;
    }
    for (int64_t c = t->child[i]; c < t->child[i] + t->nchild[i]; c++) walk(t, c, g, P, out);
}

/* Build every group's list; returns the total number of entries. */
int64_t or_lists(or_tree *t, double rcut, double theta)
{
    or_prm P = make_prm(1.0, 0.0, rcut, theta);
    int64_t G = t->n_groups;
    ivec *tmp = (ivec *)calloc((size_t)(G > 0 ? G : 1), sizeof(ivec));
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t g = 0; g < G; g++)
        if (t->n_nodes > 0) walk(t, 0, g, &P, &tmp[g]);
    free(t->loff);
    free(t->ent);
    t->loff = (int64_t *)malloc(sizeof(int64_t) * (size_t)(G + 1));
    t->loff[0] = 0;
    for (int64_t g = 0; g < G; g++) t->loff[g + 1] = t->loff[g] + tmp[g].n;
    t->n_entries = t->loff[G];
    t->ent = (int64_t *)malloc(sizeof(int64_t) * (size_t)(t->n_entries > 0 ? t->n_entries : 1));
    for (int64_t g = 0; g < G; g++) {
        if (tmp[g].n) memcpy(t->ent + t->loff[g], tmp[g].v, sizeof(int64_t) * (size_t)tmp[g].n);
        free(tmp[g].v);
    }
    free(tmp);
    return t->n_entries;
}

/* Positions of an entry (particle or node monopole) and its mass. */
static inline void entry_src(const or_tree *t, int64_t e, double *xj, double *mj)
{
    if (e >= 0) {
        for (int k = 0; k < 3; k++) xj[k] = t->xb[k][e];
        *mj = t->m[e];
    } else {
        int64_t nd = -e - 1;
        for (int k = 0; k < 3; k++) xj[k] = t->com[k][nd];
        *mj = t->M[nd];
    }
}

/* Eq. 2 over the lists of groups [g0, g1) (nodes enter as monopoles, the self
 * entry is skipped); acc is written in input order for those groups' particles. */
void or_list_forces_range(const or_tree *t, int64_t g0, int64_t g1, double G, double eps,
                          double rcut, double *acc, int xi_soft)
{
    or_prm P = make_prm_xi(G, eps, rcut, xi_soft);
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t g = g0; g < g1; g++) {
        for (int64_t i = t->gfirst[g]; i < t->gfirst[g] + t->gcount[g]; i++) {
            double ax = 0, ay = 0, az = 0;
            for (int64_t q = t->loff[g]; q < t->loff[g + 1]; q++) {
                int64_t e = t->ent[q];
                if (e == i) continue;
                double xj[3], mj;
                entry_src(t, e, xj, &mj);
                pair_acc(minimg(xj[0] - t->xb[0][i]), minimg(xj[1] - t->xb[1][i]),
                         minimg(xj[2] - t->xb[2][i]), mj, &P, &ax, &ay, &az);
            }
            int64_t o = t->perm[i];
            acc[3 * o] = ax; acc[3 * o + 1] = ay; acc[3 * o + 2] = az;
        }
    }
}

void or_list_forces(const or_tree *t, double G, double eps, double rcut, double *acc,
                    int xi_soft)
{
    or_list_forces_range(t, 0, t->n_groups, G, eps, rcut, acc, xi_soft);
}

/* sum over the groups groups[0..ng) of sum_i w_i . a_i, a_i the list force of
 * or_list_forces (input-order w): the part of a loss linear in the
 * accelerations that the listed groups carry.  Central differences of a
 * frozen tree need only the groups whose lists see the moved particle. */
double or_list_loss_groups(const or_tree *t, const int64_t *groups, int64_t ng, double G, double eps,
                           double rcut, const double *wv, int xi_soft)
{
    or_prm P = make_prm_xi(G, eps, rcut, xi_soft);
    double total = 0.0;
    for (int64_t q = 0; q < ng; q++) {
        int64_t g = groups[q];
        for (int64_t i = t->gfirst[g]; i < t->gfirst[g] + t->gcount[g]; i++) {
            double ax = 0, ay = 0, az = 0;
            for (int64_t e2 = t->loff[g]; e2 < t->loff[g + 1]; e2++) {
                int64_t e = t->ent[e2];
                if (e == i) continue;
                double xj[3], mj;
                entry_src(t, e, xj, &mj);
                pair_acc(minimg(xj[0] - t->xb[0][i]), minimg(xj[1] - t->xb[1][i]),
                         minimg(xj[2] - t->xb[2][i]), mj, &P, &ax, &ay, &az);
            }
            const double *w = wv + 3 * t->perm[i];
            total += (w[0] * ax + w[1] * ay) + w[2] * az;
        }
    }
    return total;
}

/* Pairs of the lists whose Eq. 2 term is not identically zero: over every
 * group, every member particle i and every list entry (particle or monopole)
 * other than i itself, count the pair when its distance r is positive and its
 * cutoff distance -- r, or s = sqrt(r^2 + eps^2) in the softened-xi variant --
 * is below r_cut (Eq. 3 vanishes at and beyond the cutoff).  The sum over
 * groups of n_i * n_j counts every evaluated pair; this counts the useful ones
 * among them.  The decision is taken in FP64 exactly as pair_acc takes it. */
int64_t or_count_useful(const or_tree *t, double eps, double rcut, int xi_soft)
{
    or_prm P = make_prm_xi(1.0, eps, rcut, xi_soft);
    int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 8) reduction(+ : total)
    for (int64_t g = 0; g < t->n_groups; g++) {
        for (int64_t i = t->gfirst[g]; i < t->gfirst[g] + t->gcount[g]; i++) {
            for (int64_t q = t->loff[g]; q < t->loff[g + 1]; q++) {
                int64_t e = t->ent[q];
                if (e == i) continue;
                double xj[3], mj;
                entry_src(t, e, xj, &mj);
                double dx = minimg(xj[0] - t->xb[0][i]);
                double dy = minimg(xj[1] - t->xb[1][i]);
                double dz = minimg(xj[2] - t->xb[2][i]);
                double r2 = (dx * dx + dy * dy) + dz * dz;
                if (r2 == 0.0) continue;
                double c2 = P.soft ? r2 + P.eps2 : r2;
                if (c2 < P.rc2) total++;
            }
        }
    }
    return total;
}

/* Vector-Jacobian product of or_list_forces for fixed lists: w = dL/da (input
 * order) -> dL/dx (input order).  Per pair v = G m_j J(d) w_i goes to -i and +j;
 * for a node entry it goes to the node's cotangent c_n, which reaches each
 * member p as m_p * sum over the ancestors a of p of c_a / M_a (the derivative
 * of the centre of mass). */
void or_list_vjp_range(const or_tree *t, int64_t g0, int64_t g1, double G, double eps,
                       double rcut, const double *wv, double *grad, int xi_soft)
{
    or_prm P = make_prm_xi(G, eps, rcut, xi_soft);
    int64_t n = t->n, nn = t->n_nodes;
    double *gs = (double *)calloc((size_t)(3 * (n > 0 ? n : 1)), sizeof(double));
    double *cot = (double *)calloc((size_t)(3 * (nn > 0 ? nn : 1)), sizeof(double));
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t g = g0; g < g1; g++) {
        for (int64_t i = t->gfirst[g]; i < t->gfirst[g] + t->gcount[g]; i++) {
            const double *wi = wv + 3 * t->perm[i];
            double gi[3] = {0, 0, 0};
            for (int64_t q = t->loff[g]; q < t->loff[g + 1]; q++) {
                int64_t e = t->ent[q];
                if (e == i) continue;
                double xj[3], mj, v[3];
                entry_src(t, e, xj, &mj);
                pair_jw(minimg(xj[0] - t->xb[0][i]), minimg(xj[1] - t->xb[1][i]),
                        minimg(xj[2] - t->xb[2][i]), mj, wi, &P, v);
                for (int k = 0; k < 3; k++) gi[k] -= v[k];
                double *dst = e >= 0 ? gs + 3 * e : cot + 3 * (-e - 1);
                for (int k = 0; k < 3; k++) {
#pragma omp atomic
                    dst[k] += v[k];
                }
            }
            for (int k = 0; k < 3; k++) {
#pragma omp atomic
                gs[3 * i + k] += gi[k];
            }
        }
    }
    /* push node cotangents down to the particles: prefix over ancestors */
    double *pre = (double *)calloc((size_t)(3 * (nn > 0 ? nn : 1)), sizeof(double));
    for (int64_t i = 0; i < nn; i++) {
        for (int k = 0; k < 3; k++) {
            double own = t->M[i] > 0.0 ? cot[3 * i + k] / t->M[i] : 0.0;
            pre[3 * i + k] = (t->parent[i] >= 0 ? pre[3 * t->parent[i] + k] : 0.0) + own;
        }
    }
    for (int64_t i = 0; i < nn; i++) {
        if (!is_leaf(t, i)) continue;
        for (int64_t p = t->first[i]; p < t->first[i] + t->count[i]; p++)
            for (int k = 0; k < 3; k++) gs[3 * p + k] += t->m[p] * pre[3 * i + k];
    }
    for (int64_t p = 0; p < n; p++)
        for (int k = 0; k < 3; k++) grad[3 * t->perm[p] + k] = gs[3 * p + k];
    free(pre);
    free(cot);
    free(gs);
}

/* The gradient of sum_i w_i . a_i for all groups' lists. */
void or_list_vjp(const or_tree *t, double G, double eps, double rcut, const double *wv,
                 double *grad, int xi_soft)
{
    or_list_vjp_range(t, 0, t->n_groups, G, eps, rcut, wv, grad, xi_soft);
}

/* Re-take the monopoles from new positions (input order) with the tree, the
 * groups and the lists frozen: each particle keeps the periodic image nearest
 * to where it was when the tree was built.  Used for finite differences. */
void or_refresh_moments(or_tree *t, const double *pos)
{
    for (int64_t s = 0; s < t->n; s++) {
        int64_t i = t->perm[s];
        for (int c = 0; c < 3; c++) t->xb[c][s] = t->x[c][s] + minimg(pos[3 * i + c] - t->x[c][s]);
    }
    moments(t, 0);
}

/* ------------------------------------------------------------------------ */
/* Export                                                                   */
/* ------------------------------------------------------------------------ */
void or_sizes(const or_tree *t, int64_t *out)
{
    out[0] = t->n; out[1] = t->n_nodes; out[2] = t->n_groups; out[3] = t->n_entries;
}

/* keys[n], perm[n] */
void or_export_keys(const or_tree *t, uint64_t *keys, int64_t *perm)
{
    if (t->n) {
        memcpy(keys, t->key, sizeof(uint64_t) * (size_t)t->n);
        memcpy(perm, t->perm, sizeof(int64_t) * (size_t)t->n);
    }
}

/* per node: ints [level, first, count, child, nchild, parent];
 * doubles [M, com xyz, lo xyz, hi xyz, cen xyz, half xyz] (16 per node) */
void or_export_nodes(const or_tree *t, int64_t *ints, double *dbl)
{
    for (int64_t i = 0; i < t->n_nodes; i++) {
        int64_t *a = ints + 6 * i;
        a[0] = t->level[i]; a[1] = t->first[i]; a[2] = t->count[i];
        a[3] = t->child[i]; a[4] = t->nchild[i]; a[5] = t->parent[i];
        double *d = dbl + 16 * i;
        d[0] = t->M[i];
        for (int c = 0; c < 3; c++) {
            d[1 + c] = t->com[c][i]; d[4 + c] = t->lo[c][i]; d[7 + c] = t->hi[c][i];
            d[10 + c] = t->cen[c][i]; d[13 + c] = t->half[c][i];
        }
    }
}

/* per group: ints [first, count]; doubles [cen xyz, half xyz] */
void or_export_groups(const or_tree *t, int64_t *ints, double *dbl)
{
    for (int64_t g = 0; g < t->n_groups; g++) {
        ints[2 * g] = t->gfirst[g]; ints[2 * g + 1] = t->gcount[g];
        for (int c = 0; c < 3; c++) { dbl[6 * g + c] = t->gc[c][g]; dbl[6 * g + 3 + c] = t->gh[c][g]; }
    }
}

void or_export_lists(const or_tree *t, int64_t *loff, int64_t *ent)
{
    memcpy(loff, t->loff, sizeof(int64_t) * (size_t)(t->n_groups + 1));
    if (t->n_entries) memcpy(ent, t->ent, sizeof(int64_t) * (size_t)t->n_entries);
}

void or_free(or_tree *t)
{
    if (!t) return;
    free(t->key); free(t->perm); free(t->m);
    for (int c = 0; c < 3; c++) {
        free(t->x[c]); free(t->xb[c]);
        free(t->S[c]); free(t->com[c]); free(t->lo[c]); free(t->hi[c]);
        free(t->cen[c]); free(t->half[c]); free(t->gc[c]); free(t->gh[c]);
    }
    free(t->level); free(t->first); free(t->count); free(t->child); free(t->nchild);
    free(t->parent); free(t->M); free(t->gfirst); free(t->gcount);
    free(t->loff); free(t->ent);
    free(t);
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
