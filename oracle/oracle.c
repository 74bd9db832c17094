/*
 * oracle.c -- plain FP64 CPU reference for softened gravity, direct and octree.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * timed CPU-baseline leg of the benchmark may load this file's library.  It
 * shares no code, header or constant table with the GPU path; both sides read
 * the same seeded inputs and nothing else.
 *
 * What it computes (paper: Section II "Octree Method", II-A "Tree
 * Representation", II-B "MAC Condition", III-B/III-C tree construction and
 * cell properties, III-D vectorised group walk):
 *
 *   oracle_direct      Plummer-softened direct sum, j != i excluded.  The paper
 *                      never prints the pair law; it only says particles carry a
 *                      softening length (Section III-D).  Reading: a_i = sum_j
 *                      m_j (x_j - x_i) / (|x_j - x_i|^2 + eps^2)^(3/2),
 *                      phi_i = -sum_j m_j / (|x_j - x_i|^2 + eps^2)^(1/2), G = 1.
 *   oracle_cell_*      monopole (Section II, p = 1) and, as an extension, the
 *                      traceless quadrupole about the centre of mass; the cell's
 *                      field is evaluated with the same softening.
 *   oracle_tree_*      pointer-free recursive octree on a 2^21 grid per axis,
 *                      leaves of at most leaf_size particles, groups = maximal
 *                      cells with at most n_crit particles, one shared walk per
 *                      group with a group MAC -- the opening angle, or the
 *                      Salmon-Warren absolute MAC of Section II-B (Eq. SW_MAC
 *                      with B_2 of Eq. B2 and the m_limit rule of Section
 *                      III-C) -- forces summed over the walk's cell and
 *                      particle entries.
 *   oracle_tree_features  the five list statistics of each group that feed
 *                      the learned opening angle (a reading of this
 *                      project: the paper's accuracy control is Delta).
 *   oracle_sw_radius   B_2, b_max and the bounding radius r_b of one particle
 *                      set (Eq. B2, Eq. SW_MAC).
 *   oracle_sph_*       SPH sums (Section II, "Bounding Radius for SPH"): the
 *                      density rho_i = sum_j m_j W(|x_i - x_j|, h_j) (Eq.
 *                      SPH_SUM with A = m) by direct summation and by the
 *                      group walk with the bounding radius r_SPH of Eq.
 *                      SPH_RAD (cells whose sphere misses the group box are
 *                      skipped; particles of the other leaves are summed).
 *                      Readings: the M4 cubic spline with support radius h
 *                      (the paper: W is bell-shaped and vanishes beyond h),
 *                      scatter form (each source's own h_j, as r_SPH uses
 *                      it), the source itself included.
 *
 * Everything is written for a reader to check by eye: no blocking, no fusion,
 * summation in plain loops.  Compile with -ffp-contract=off so that no FMA
 * contraction changes the rounding of the tree geometry between machines.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_LEVELS 21                 /* 2^21 grid cells per axis (63-bit keys) */
#define ORACLE_GRID   2097152.0          /* 2^21 */
#define ORACLE_PI     3.14159265358979323846

/* ------------------------------------------------------------------------- */
/* C1: direct sum (reading of Section II: particle-particle interaction).     */
/* ------------------------------------------------------------------------- */

/* Pair law for one source at offset (dx,dy,dz) = x_j - x_i. */
static void pair_mono(double dx, double dy, double dz, double m, double eps2,
                      double acc[3], double* pot)
{
    double r2 = dx * dx + dy * dy + dz * dz + eps2;
    double rinv = 1.0 / sqrt(r2);
    double rinv3 = rinv * rinv * rinv;
    acc[0] += m * rinv3 * dx;
    acc[1] += m * rinv3 * dy;
    acc[2] += m * rinv3 * dz;
    *pot -= m * rinv;
}

/*
 * Direct sum for the targets tgt[0..n_tgt) (indices into the source arrays)
 * against all n_src sources, skipping the source with the target's own index.
 * pos: [n_src][3], mass: [n_src]; acc: [n_tgt][3], pot: [n_tgt].
 */
int oracle_direct(int64_t n_src, const double* pos, const double* mass,
                  int64_t n_tgt, const int64_t* tgt, double eps,
                  double* acc, double* pot)
{
    if (n_src < 0 || n_tgt < 0 || !(eps > 0.0)) return -1;
    double eps2 = eps * eps;
    int64_t t;
#pragma omp parallel for schedule(dynamic, 4)
    for (t = 0; t < n_tgt; ++t) {
        int64_t i = tgt[t];
        double a[3] = {0.0, 0.0, 0.0};
        double p = 0.0;
        for (int64_t j = 0; j < n_src; ++j) {
            if (j == i) continue;
            pair_mono(pos[3 * j] - pos[3 * i], pos[3 * j + 1] - pos[3 * i + 1],
                      pos[3 * j + 2] - pos[3 * i + 2], mass[j], eps2, a, &p);
        }
        acc[3 * t] = a[0];
        acc[3 * t + 1] = a[1];
        acc[3 * t + 2] = a[2];
        pot[t] = p;
    }
    return 0;
}

/* M4 cubic spline with support radius h, normalised to unit volume in 3D:
   W = 8 / (pi h^3) * w(q), q = r / h,
   w = 1 - 6 q^2 + 6 q^3 for q <= 1/2, 2 (1 - q)^3 for 1/2 < q < 1, 0 beyond. */
static double sph_w(double r, double h)
{
    double q = r / h;
    double w;
    if (q <= 0.5)
        w = 1.0 - 6.0 * q * q + 6.0 * q * q * q;
    else if (q < 1.0)
        w = 2.0 * (1.0 - q) * (1.0 - q) * (1.0 - q);
    else
        w = 0.0;
    return 8.0 / (ORACLE_PI * h * h * h) * w;
}

int oracle_sph_kernel(double r, double h, double* w)
{
    if (!(h > 0.0) || r < 0.0) return -1;
    *w = sph_w(r, h);
    return 0;
}

/* rho[t] = sum over all sources j of m_j W(|x_i - x_j|, h_j), i = tgt[t]
   (the source i itself included). */
int oracle_sph_density_direct(int64_t n, const double* pos, const double* mass, const double* h, int64_t n_tgt,
                              const int64_t* tgt, double* rho)
{
    if (n <= 0 || n_tgt < 0) return -1;
    for (int64_t j = 0; j < n; ++j)
        if (!(h[j] > 0.0)) return -1;
    int64_t t;
#pragma omp parallel for schedule(static)
    for (t = 0; t < n_tgt; ++t) {
        int64_t i = tgt[t];
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double dx = pos[3 * j] - pos[3 * i], dy = pos[3 * j + 1] - pos[3 * i + 1], dz = pos[3 * j + 2] - pos[3 * i + 2];
            s += mass[j] * sph_w(sqrt(dx * dx + dy * dy + dz * dz), h[j]);
        }
        rho[t] = s;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Cell moments and the cell field (Section II: the cell acts as a virtual    */
/* particle at its centre of mass; the quadrupole is an extension).          */
/* ------------------------------------------------------------------------- */

/*
 * Mass, centre of mass and traceless quadrupole Q_ab = sum m (3 d_a d_b -
 * |d|^2 delta_ab), d = x - com, of the particles idx[0..n).  q is written as
 * (Qxx, Qyy, Qzz, Qxy, Qxz, Qyz).
 */
static void moments(const double* pos, const double* mass, const int64_t* idx, int64_t n,
                    double* m_out, double com[3], double q[6])
{
    double m = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        int64_t i = idx[k];
        m += mass[i];
        sx += mass[i] * pos[3 * i];
        sy += mass[i] * pos[3 * i + 1];
        sz += mass[i] * pos[3 * i + 2];
    }
    com[0] = sx / m;
    com[1] = sy / m;
    com[2] = sz / m;
    for (int c = 0; c < 6; ++c) q[c] = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        int64_t i = idx[k];
        double dx = pos[3 * i] - com[0], dy = pos[3 * i + 1] - com[1], dz = pos[3 * i + 2] - com[2];
        double d2 = dx * dx + dy * dy + dz * dz;
        q[0] += mass[i] * (3.0 * dx * dx - d2);
        q[1] += mass[i] * (3.0 * dy * dy - d2);
        q[2] += mass[i] * (3.0 * dz * dz - d2);
        q[3] += mass[i] * (3.0 * dx * dy);
        q[4] += mass[i] * (3.0 * dx * dz);
        q[5] += mass[i] * (3.0 * dy * dz);
    }
    *m_out = m;
}

/*
 * Field at x of a cell (mass m, centre of mass com, quadrupole q, B_2 =
 * sum m |x_j - com|^2).  The cell stands for its particles (Section II: a
 * cell acts as a virtual particle at its centre of mass); the quadrupole
 * term is this library's extension: the second-order Taylor term of the
 * softened pair law about the centre of mass.  With r = com - x,
 * q = (|r|^2 + eps^2)^(-1/2) and the second moment D = sum m d d^T
 * (d = x_j - com, so Q = 3 D - tr(D) I and tr(D) = B_2), the Hessian of q
 * is 3 r r^T q^5 - I q^3, and one half of its contraction with D is
 *     (1/2) (r.Q.r - B_2 eps^2) q^5.
 * The potential is therefore
 *     phi = -m q - (1/2) (r.Q.r - B_2 eps^2) q^5
 * and the acceleration a = -grad_x phi is
 *     a = m q^3 r - q^5 Q r + (5/2) (r.Q.r - B_2 eps^2) q^7 r.
 * Without softening the B_2 term vanishes (the Laplace multipole).
 * use_quad = 0 keeps the monopole only.
 */
static void cell_field(const double x[3], double m, const double com[3], const double q[6], double b2,
                       int use_quad, double eps2, double acc[3], double* pot)
{
    double rx = com[0] - x[0], ry = com[1] - x[1], rz = com[2] - x[2];
    double r2 = rx * rx + ry * ry + rz * rz + eps2;
    double rinv = 1.0 / sqrt(r2);
    double rinv2 = rinv * rinv;
    double rinv3 = rinv * rinv2;
    acc[0] += m * rinv3 * rx;
    acc[1] += m * rinv3 * ry;
    acc[2] += m * rinv3 * rz;
    *pot -= m * rinv;
    if (!use_quad) return;
    double Qr0 = q[0] * rx + q[3] * ry + q[4] * rz;
    double Qr1 = q[3] * rx + q[1] * ry + q[5] * rz;
    double Qr2 = q[4] * rx + q[5] * ry + q[2] * rz;
    double rQr = rx * Qr0 + ry * Qr1 + rz * Qr2;
    double w = rQr - b2 * eps2;
    double rinv5 = rinv3 * rinv2;
    double rinv7 = rinv5 * rinv2;
    acc[0] += -Qr0 * rinv5 + 2.5 * w * rx * rinv7;
    acc[1] += -Qr1 * rinv5 + 2.5 * w * ry * rinv7;
    acc[2] += -Qr2 * rinv5 + 2.5 * w * rz * rinv7;
    *pot -= 0.5 * w * rinv5;
}

/*
 * Spread of a particle set about its centre of mass com (Section II-B):
 * B_2 = sum m |com - x|^2 (Eq. B2, the trace of the second moment) and
 * b_max = max |com - x|.
 */
static void spread(const double* pos, const double* mass, const int64_t* idx, int64_t n, const double com[3],
                   double* b2_out, double* bmax_out)
{
    double b2 = 0.0, dmax2 = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        int64_t i = idx[k];
        double dx = com[0] - pos[3 * i], dy = com[1] - pos[3 * i + 1], dz = com[2] - pos[3 * i + 2];
        double d2 = dx * dx + dy * dy + dz * dz;
        b2 += mass[i] * d2;
        if (d2 > dmax2) dmax2 = d2;
    }
    *b2_out = b2;
    *bmax_out = sqrt(dmax2);
}

/*
 * Bounding radius of the absolute MAC (Eq. SW_MAC): the distance d at which
 * the monopole error bound 3 B_2 / (d^2 (d - b_max)^2) equals the accuracy
 * parameter delta (an acceleration),
 *     r_b = b_max / 2 + sqrt(b_max^2 / 4 + sqrt(3 B_2 / delta)).
 * A cell heavier than m_limit (> 0) gets r_b = 2 S_root, so that it is never
 * accepted (Section III-C).  delta <= 0 accepts nothing (r_b infinite).
 */
static double sw_radius(double b2, double bmax, double m, double delta, double m_limit, double s_root)
{
    if (m_limit > 0.0 && m > m_limit) return 2.0 * s_root;
    if (!(delta > 0.0)) return INFINITY;
    double h = 0.5 * bmax;
    return h + sqrt(h * h + sqrt(3.0 * b2 / delta));
}

/* Exposed for the tests: B_2, b_max and r_b of the particle set (out[0..2]). */
int oracle_sw_radius(const double* pos, const double* mass, int64_t n, double delta, double m_limit,
                     double s_root, double* out)
{
    if (n <= 0) return -1;
    int64_t* idx = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    if (!idx) return -2;
    for (int64_t k = 0; k < n; ++k) idx[k] = k;
    double m, com[3], q[6];
    moments(pos, mass, idx, n, &m, com, q);
    spread(pos, mass, idx, n, com, &out[0], &out[1]);
    free(idx);
    out[2] = sw_radius(out[0], out[1], m, delta, m_limit, s_root);
    return 0;
}

/* Exposed for the tests: moments of a particle set (mass, centre of mass,
   traceless quadrupole, B_2) and the field they make. */
int oracle_cell_moments(const double* pos, const double* mass, int64_t n,
                        double* m_out, double* com, double* q, double* b2_out)
{
    if (n <= 0) return -1;
    int64_t* idx = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    if (!idx) return -2;
    for (int64_t k = 0; k < n; ++k) idx[k] = k;
    moments(pos, mass, idx, n, m_out, com, q);
    double bmax;
    spread(pos, mass, idx, n, com, b2_out, &bmax);
    free(idx);
    return 0;
}

int oracle_cell_field(const double* x, double m, const double* com, const double* q, double b2,
                      int use_quad, double eps, double* acc, double* pot)
{
    double a[3] = {0.0, 0.0, 0.0};
    double p = 0.0;
    cell_field(x, m, com, q, b2, use_quad, eps * eps, a, &p);
    acc[0] = a[0];
    acc[1] = a[1];
    acc[2] = a[2];
    *pot = p;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Octree (Sections II, III-B, III-C).                                       */
/* ------------------------------------------------------------------------- */

typedef struct Node {
    int level;                 /* 0 = root */
    int64_t org[3];            /* integer origin of the cube on the 2^21 grid */
    int64_t begin, end;        /* slice of the tree's particle index array */
    int n_child;
    struct Node* child[8];     /* children in octant order, NULL where empty */
    double m, com[3], q[6];
    double b2, bmax;           /* spread about the centre of mass (Eq. B2) */
    double rsph;               /* SPH bounding radius (Eq. SPH_RAD), set per call */
    double cube_lo[3], side, gc[3];   /* geometry for the MAC */
} Node;

typedef struct OracleTree {
    int64_t n;
    const double* pos;         /* caller-owned, must outlive the tree */
    const double* mass;
    int64_t* idx;              /* particle indices, partitioned by the tree */
    int64_t* gx;               /* quantised coordinates [n][3] */
    double lo[3], S, h;
    int leaf_size, n_crit;
    Node* root;
    int64_t n_cells;
    /* groups: (node, sub-range) ; a leaf at maximum depth with more than
       n_crit particles is cut into chunks of n_crit ordered by index */
    int64_t n_groups, cap_groups;
    int64_t* grp_begin;
    int64_t* grp_end;
} OracleTree;

static int cmp_i64(const void* a, const void* b)
{
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return (x > y) - (x < y);
}

static void set_geometry(OracleTree* t, Node* c)
{
    double l = t->h * (double)((int64_t)1 << (ORACLE_LEVELS - c->level));
    for (int a = 0; a < 3; ++a) {
        c->cube_lo[a] = t->lo[a] + (double)c->org[a] * t->h;
        c->gc[a] = c->cube_lo[a] + 0.5 * l;
    }
    c->side = l;
}

/* Recursive subdivision: split while count > leaf_size and level < 21. */
static Node* build_node(OracleTree* t, int level, const int64_t org[3], int64_t begin, int64_t end,
                        int64_t* scratch)
{
    Node* c = (Node*)calloc(1, sizeof(Node));
    if (!c) return NULL;
    t->n_cells++;
    c->level = level;
    c->org[0] = org[0];
    c->org[1] = org[1];
    c->org[2] = org[2];
    c->begin = begin;
    c->end = end;
    set_geometry(t, c);
    moments(t->pos, t->mass, t->idx + begin, end - begin, &c->m, c->com, c->q);
    spread(t->pos, t->mass, t->idx + begin, end - begin, c->com, &c->b2, &c->bmax);
    int64_t count = end - begin;
    if (count <= t->leaf_size || level == ORACLE_LEVELS) return c;

    /* octant of each particle: bit (20 - level) of each quantised coordinate;
       x is bit 0 of the octant, y bit 1, z bit 2 */
    int shift = ORACLE_LEVELS - 1 - level;
    int64_t counts[8] = {0};
    for (int64_t k = begin; k < end; ++k) {
        int64_t i = t->idx[k];
        int o = (int)(((t->gx[3 * i] >> shift) & 1) | (((t->gx[3 * i + 1] >> shift) & 1) << 1) |
                      (((t->gx[3 * i + 2] >> shift) & 1) << 2));
        counts[o]++;
    }
    int64_t start[8];
    int64_t s = begin;
    for (int o = 0; o < 8; ++o) {
        start[o] = s;
        s += counts[o];
    }
    int64_t fill[8];
    memcpy(fill, start, sizeof(fill));
    for (int64_t k = begin; k < end; ++k) {
        int64_t i = t->idx[k];
        int o = (int)(((t->gx[3 * i] >> shift) & 1) | (((t->gx[3 * i + 1] >> shift) & 1) << 1) |
                      (((t->gx[3 * i + 2] >> shift) & 1) << 2));
        scratch[fill[o]++] = i;
    }
    memcpy(t->idx + begin, scratch + begin, (size_t)count * sizeof(int64_t));
    int64_t half = (int64_t)1 << shift;
    for (int o = 0; o < 8; ++o) {
        if (counts[o] == 0) continue;
        int64_t corg[3] = {org[0] + ((o & 1) ? half : 0), org[1] + ((o & 2) ? half : 0),
                           org[2] + ((o & 4) ? half : 0)};
        Node* ch = build_node(t, level + 1, corg, start[o], start[o] + counts[o], scratch);
        if (!ch) return NULL;
        c->child[c->n_child++] = ch;
    }
    return c;
}

static int add_group(OracleTree* t, int64_t b, int64_t e)
{
    if (t->n_groups == t->cap_groups) {
        int64_t cap = t->cap_groups ? 2 * t->cap_groups : 1024;
        int64_t* nb = (int64_t*)realloc(t->grp_begin, (size_t)cap * sizeof(int64_t));
        if (!nb) return -1;
        t->grp_begin = nb;
        int64_t* ne = (int64_t*)realloc(t->grp_end, (size_t)cap * sizeof(int64_t));
        if (!ne) return -1;
        t->grp_end = ne;
        t->cap_groups = cap;
    }
    t->grp_begin[t->n_groups] = b;
    t->grp_end[t->n_groups] = e;
    t->n_groups++;
    return 0;
}

/* Groups: maximal cells holding at most n_crit particles. */
static int find_groups(OracleTree* t, Node* c)
{
    int64_t count = c->end - c->begin;
    if (count <= t->n_crit) return add_group(t, c->begin, c->end);
    if (c->n_child == 0) {
        /* a leaf at maximum depth with more than n_crit particles: chunks of
           n_crit in increasing particle index */
        qsort(t->idx + c->begin, (size_t)count, sizeof(int64_t), cmp_i64);
        for (int64_t b = c->begin; b < c->end; b += t->n_crit) {
            int64_t e = b + t->n_crit < c->end ? b + t->n_crit : c->end;
            if (add_group(t, b, e)) return -1;
        }
        return 0;
    }
    for (int k = 0; k < c->n_child; ++k)
        if (find_groups(t, c->child[k])) return -1;
    return 0;
}

static void free_node(Node* c)
{
    if (!c) return;
    for (int k = 0; k < c->n_child; ++k) free_node(c->child[k]);
    free(c);
}

void oracle_tree_free(void* handle)
{
    OracleTree* t = (OracleTree*)handle;
    if (!t) return;
    free_node(t->root);
    free(t->idx);
    free(t->gx);
    free(t->grp_begin);
    free(t->grp_end);
    free(t);
}

/*
 * Build the octree of n particles.  Root cube (Section III-B, first step):
 * centred on the bounding-box centre, side S = max extent * (1 + 1e-12)
 * (S = 1 when all particles coincide).  Quantised coordinate on the 2^21 grid:
 * g = floor((x - lo) * (2^21 / S)) clamped to [0, 2^21 - 1], lo = centre - S/2;
 * the octant test of every level reads one bit of g, which is the test
 * "x >= cell centre" decided on the grid.
 * Returns an opaque handle (NULL on error).  pos and mass must outlive it.
 */
void* oracle_tree_new(int64_t n, const double* pos, const double* mass, int leaf_size, int n_crit)
{
    if (n <= 0 || leaf_size < 1 || n_crit < 1) return NULL;
    OracleTree* t = (OracleTree*)calloc(1, sizeof(OracleTree));
    if (!t) return NULL;
    t->n = n;
    t->pos = pos;
    t->mass = mass;
    t->leaf_size = leaf_size;
    t->n_crit = n_crit;
    double mn[3], mx[3];
    for (int a = 0; a < 3; ++a) mn[a] = mx[a] = pos[a];
    for (int64_t i = 1; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            if (pos[3 * i + a] < mn[a]) mn[a] = pos[3 * i + a];
            if (pos[3 * i + a] > mx[a]) mx[a] = pos[3 * i + a];
        }
    double ext = 0.0;
    for (int a = 0; a < 3; ++a)
        if (mx[a] - mn[a] > ext) ext = mx[a] - mn[a];
    t->S = ext * (1.0 + 1e-12);
    if (!(t->S > 0.0)) t->S = 1.0;
    for (int a = 0; a < 3; ++a) t->lo[a] = (mn[a] + mx[a]) * 0.5 - 0.5 * t->S;
    t->h = t->S / ORACLE_GRID;
    double scale = ORACLE_GRID / t->S;

    t->idx = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    t->gx = (int64_t*)malloc((size_t)n * 3 * sizeof(int64_t));
    int64_t* scratch = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    if (!t->idx || !t->gx || !scratch) {
        free(scratch);
        oracle_tree_free(t);
        return NULL;
    }
    for (int64_t i = 0; i < n; ++i) {
        t->idx[i] = i;
        for (int a = 0; a < 3; ++a) {
            double g = floor((pos[3 * i + a] - t->lo[a]) * scale);
            if (g < 0.0) g = 0.0;
            if (g > ORACLE_GRID - 1.0) g = ORACLE_GRID - 1.0;
            t->gx[3 * i + a] = (int64_t)g;
        }
    }
    int64_t org[3] = {0, 0, 0};
    t->root = build_node(t, 0, org, 0, n, scratch);
    free(scratch);
    if (!t->root || find_groups(t, t->root)) {
        oracle_tree_free(t);
        return NULL;
    }
    return t;
}

int64_t oracle_tree_n_groups(const void* handle) { return ((const OracleTree*)handle)->n_groups; }
int64_t oracle_tree_n_cells(const void* handle) { return ((const OracleTree*)handle)->n_cells; }

/* Acceptance rule of a walk: kind 0 = opening angle theta, kind 1 = the
   Salmon-Warren absolute MAC with accuracy delta and the m_limit rule. */
typedef struct Mac {
    int kind;
    double theta;
    double delta, m_limit, s_root;
} Mac;

/* The group MAC (Barnes 1990 vectorised walk, Section III-D; notation of
   Section II-B), with d_min the distance from the cell's centre of mass to
   the group box [blo, bhi]:
   kind 0: accept cell c iff the cube does not overlap the box and
           d_min > l / theta + s (s: distance from the centre of mass to the
           cube's geometric centre);
   kind 1: accept iff d_min > r_b (Eq. SW_MAC).  No particle of the group
           can lie in such a cell: r_b >= b_max. */
static int accept(const Node* c, const double blo[3], const double bhi[3], const Mac* mac)
{
    if (mac->kind == 1) {
        double d2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            double d = 0.0;
            if (blo[a] - c->com[a] > d) d = blo[a] - c->com[a];
            if (c->com[a] - bhi[a] > d) d = c->com[a] - bhi[a];
            d2 += d * d;
        }
        return sqrt(d2) > sw_radius(c->b2, c->bmax, c->m, mac->delta, mac->m_limit, mac->s_root);
    }
    double theta = mac->theta;
    if (!(theta > 0.0)) return 0;
    int overlap = 1;
    for (int a = 0; a < 3; ++a) {
        double clo = c->cube_lo[a], chi = c->cube_lo[a] + c->side;
        if (!(clo <= bhi[a] && blo[a] <= chi)) overlap = 0;
    }
    if (overlap) return 0;
    double d2 = 0.0, s2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        double d = 0.0;
        if (blo[a] - c->com[a] > d) d = blo[a] - c->com[a];
        if (c->com[a] - bhi[a] > d) d = c->com[a] - bhi[a];
        d2 += d * d;
        double e = c->com[a] - c->gc[a];
        s2 += e * e;
    }
    return sqrt(d2) > c->side / theta + sqrt(s2);
}

/* Exposed for the tests: the opening-angle decision (kind 0 above) for one
   cell given by its cube (lower corner cube_lo, side) and centre of mass
   com, against the group box [blo, bhi].  The cube centre is cube_lo +
   side / 2.  *out = 1 accept, 0 open. */
int oracle_group_mac(const double* cube_lo, double side, const double* com, const double* blo, const double* bhi,
                     double theta, int* out)
{
    if (!(side > 0.0) || !(theta >= 0.0) || !out) return -1;
    Node c;
    memset(&c, 0, sizeof(c));
    for (int a = 0; a < 3; ++a) {
        c.cube_lo[a] = cube_lo[a];
        c.com[a] = com[a];
        c.gc[a] = cube_lo[a] + side / 2.0;
    }
    c.side = side;
    Mac mac;
    memset(&mac, 0, sizeof(mac));
    mac.kind = 0;
    mac.theta = theta;
    *out = accept(&c, blo, bhi, &mac);
    return 0;
}

typedef struct Entries {
    int64_t n_cell, n_part, cap_cell, cap_part;
    const Node** cell;
    int64_t* part;
} Entries;

static int push_cell(Entries* e, const Node* c)
{
    if (e->n_cell == e->cap_cell) {
        int64_t cap = e->cap_cell ? 2 * e->cap_cell : 256;
        const Node** nc = (const Node**)realloc((void*)e->cell, (size_t)cap * sizeof(Node*));
        if (!nc) return -1;
        e->cell = nc;
        e->cap_cell = cap;
    }
    e->cell[e->n_cell++] = c;
    return 0;
}

static int push_part(Entries* e, int64_t i)
{
    if (e->n_part == e->cap_part) {
        int64_t cap = e->cap_part ? 2 * e->cap_part : 1024;
        int64_t* np = (int64_t*)realloc(e->part, (size_t)cap * sizeof(int64_t));
        if (!np) return -1;
        e->part = np;
        e->cap_part = cap;
    }
    e->part[e->n_part++] = i;
    return 0;
}

/* The walk (Section II-A rules (1)-(4), written recursively): an accepted
   cell becomes one cell entry; a rejected cell opens into its children; a
   rejected leaf contributes each of its particles. */
static int walk(const OracleTree* t, const Node* c, const double blo[3], const double bhi[3],
                const Mac* mac, Entries* e)
{
    if (accept(c, blo, bhi, mac)) return push_cell(e, c);
    if (c->n_child == 0) {
        for (int64_t k = c->begin; k < c->end; ++k)
            if (push_part(e, t->idx[k])) return -1;
        return 0;
    }
    for (int k = 0; k < c->n_child; ++k)
        if (walk(t, c->child[k], blo, bhi, mac, e)) return -1;
    return 0;
}

/*
 * Evaluate the tree force.  For each group (every group_stride-th one, in the
 * tree's own order) walk the tree with the group MAC and sum the pair law
 * over particle entries (j != i) and the cell field over cell entries.
 * mac_kind 0: opening angle; theta_by_key, if not NULL, gives the group's
 * angle at the index of its lowest-numbered particle (length n), otherwise
 * theta is used.  mac_kind 1: the absolute MAC with accuracy delta and mass
 * limit m_limit (<= 0: none); theta and theta_by_key are not used.
 * Outputs in the caller's particle order: acc [n][3], pot [n]; entries of
 * particles in skipped groups are left untouched.
 * Per-group statistics (arrays of length n_groups, any may be NULL):
 *   g_key    lowest particle index in the group,   g_count  particles,
 *   g_ncell  cell entries,  g_npart  particle entries,
 *   g_mass   mass of all entries (equals the total mass when the walk is complete).
 * *interactions receives sum over evaluated groups of count * (ncell + npart).
 * group_sel (n_sel entries, group indices), if not NULL, replaces the
 * stride: only those groups are walked and evaluated (the statistics of the
 * other groups are left untouched), so that a sample of groups costs what
 * its own walks and sums cost.
 */
int oracle_tree_eval(const void* handle, double theta, const double* theta_by_key, int mac_kind, double delta,
                     double m_limit, double eps, int use_quad, int64_t group_stride, const int64_t* group_sel,
                     int64_t n_sel, double* acc, double* pot, int64_t* g_key, int64_t* g_count, int64_t* g_ncell,
                     int64_t* g_npart, double* g_mass, int64_t* interactions)
{
    const OracleTree* t = (const OracleTree*)handle;
    if (!t || !(eps > 0.0) || group_stride < 1 || mac_kind < 0 || mac_kind > 1) return -1;
    if (group_sel) {
        if (n_sel < 0) return -1;
        for (int64_t q = 0; q < n_sel; ++q)
            if (group_sel[q] < 0 || group_sel[q] >= t->n_groups) return -1;
    }
    const int64_t n_loop = group_sel ? n_sel : t->n_groups;
    double eps2 = eps * eps;
    int64_t total = 0;
    int err = 0;
    int64_t q;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total) reduction(| : err)
    for (q = 0; q < n_loop; ++q) {
        const int64_t g = group_sel ? group_sel[q] : q;
        const int evaluate = group_sel ? 1 : (g % group_stride == 0);
        int64_t b = t->grp_begin[g], e_ = t->grp_end[g];
        double blo[3], bhi[3];
        int64_t key = t->idx[b];
        for (int a = 0; a < 3; ++a) blo[a] = bhi[a] = t->pos[3 * t->idx[b] + a];
        for (int64_t k = b; k < e_; ++k) {
            int64_t i = t->idx[k];
            if (i < key) key = i;
            for (int a = 0; a < 3; ++a) {
                if (t->pos[3 * i + a] < blo[a]) blo[a] = t->pos[3 * i + a];
                if (t->pos[3 * i + a] > bhi[a]) bhi[a] = t->pos[3 * i + a];
            }
        }
        Mac mac;
        mac.kind = mac_kind;
        mac.theta = theta_by_key ? theta_by_key[key] : theta;
        mac.delta = delta;
        mac.m_limit = m_limit;
        mac.s_root = t->S;
        Entries ent;
        memset(&ent, 0, sizeof(ent));
        if (walk(t, t->root, blo, bhi, &mac, &ent)) {
            err |= 1;
            free((void*)ent.cell);
            free(ent.part);
            continue;
        }
        if (g_key) g_key[g] = key;
        if (g_count) g_count[g] = e_ - b;
        if (g_ncell) g_ncell[g] = ent.n_cell;
        if (g_npart) g_npart[g] = ent.n_part;
        if (g_mass) {
            double ms = 0.0;
            for (int64_t k = 0; k < ent.n_cell; ++k) ms += ent.cell[k]->m;
            for (int64_t k = 0; k < ent.n_part; ++k) ms += t->mass[ent.part[k]];
            g_mass[g] = ms;
        }
        if (evaluate) {
            total += (e_ - b) * (ent.n_cell + ent.n_part);
            for (int64_t k = b; k < e_; ++k) {
                int64_t i = t->idx[k];
                const double* xi = t->pos + 3 * i;
                double a[3] = {0.0, 0.0, 0.0};
                double p = 0.0;
                for (int64_t c = 0; c < ent.n_cell; ++c) {
                    const Node* cn = ent.cell[c];
                    cell_field(xi, cn->m, cn->com, cn->q, cn->b2, use_quad, eps2, a, &p);
                }
                for (int64_t c = 0; c < ent.n_part; ++c) {
                    int64_t j = ent.part[c];
                    if (j == i) continue;
                    pair_mono(t->pos[3 * j] - xi[0], t->pos[3 * j + 1] - xi[1],
                              t->pos[3 * j + 2] - xi[2], t->mass[j], eps2, a, &p);
                }
                acc[3 * i] = a[0];
                acc[3 * i + 1] = a[1];
                acc[3 * i + 2] = a[2];
                pot[i] = p;
            }
        }
        free((void*)ent.cell);
        free(ent.part);
    }
    if (interactions) *interactions = total;
    return err ? -2 : 0;
}

/*
 * List statistics of each group for the learned opening angle (a reading of
 * this project, not of the paper: the paper controls accuracy by Delta,
 * Section II-B).  The group walks the tree with opening angle theta; with
 * [blo, bhi] its particles' box, c = (blo + bhi) / 2, eps the softening and
 * d_c the distance from cell c's centre of mass to the box:
 *   f0 = log2 max(1, n_cell + n_part)                (list length)
 *   f1 = log10 max(min over cells of d_c / l_c, 1e-3), 3 without cells
 *   f2 = log10 (max(h, 1e-3 eps) / eps), h = half the box diagonal
 *   f3 = cell mass / mass of all entries (0 when that is 0)
 *   f4 = log10 max(T / max(|A|, 1e-300), 1e-12) with T = sum over cells of
 *        B_2 b_max / max(d_c, 1e-300)^5 (Eq. B2) and A = sum over all
 *        entries of m (x - c) / (|x - c|^2 + eps^2)^(3/2), x the entry's
 *        position (a cell's centre of mass).
 * g_key[g] receives the group's lowest particle index, feat[5 g + k] = f_k.
 */
int oracle_tree_features(const void* handle, double theta, double eps, int64_t* g_key, double* feat)
{
    const OracleTree* t = (const OracleTree*)handle;
    if (!t || !(eps > 0.0) || !(theta >= 0.0) || !g_key || !feat) return -1;
    int err = 0;
    int64_t g;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
    for (g = 0; g < t->n_groups; ++g) {
        int64_t b = t->grp_begin[g], e_ = t->grp_end[g];
        double blo[3], bhi[3];
        int64_t key = t->idx[b];
        for (int a = 0; a < 3; ++a) blo[a] = bhi[a] = t->pos[3 * t->idx[b] + a];
        for (int64_t k = b; k < e_; ++k) {
            int64_t i = t->idx[k];
            if (i < key) key = i;
            for (int a = 0; a < 3; ++a) {
                if (t->pos[3 * i + a] < blo[a]) blo[a] = t->pos[3 * i + a];
                if (t->pos[3 * i + a] > bhi[a]) bhi[a] = t->pos[3 * i + a];
            }
        }
        Mac mac;
        memset(&mac, 0, sizeof(mac));
        mac.kind = 0;
        mac.theta = theta;
        Entries ent;
        memset(&ent, 0, sizeof(ent));
        if (walk(t, t->root, blo, bhi, &mac, &ent)) {
            err |= 1;
            free((void*)ent.cell);
            free(ent.part);
            continue;
        }
        double c[3], diag2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            c[a] = 0.5 * (blo[a] + bhi[a]);
            diag2 += (bhi[a] - blo[a]) * (bhi[a] - blo[a]);
        }
        double h = 0.5 * sqrt(diag2);
        if (h < 1e-3 * eps) h = 1e-3 * eps;
        double A[3] = {0.0, 0.0, 0.0};
        double m_cells = 0.0, m_all = 0.0, T = 0.0, min_ratio = 1e3;
        for (int64_t k = 0; k < ent.n_cell + ent.n_part; ++k) {
            const int is_cell = k < ent.n_cell;
            const Node* cn = is_cell ? ent.cell[k] : NULL;
            const double* x = is_cell ? cn->com : t->pos + 3 * ent.part[k - ent.n_cell];
            const double m = is_cell ? cn->m : t->mass[ent.part[k - ent.n_cell]];
            double r2 = 0.0, r[3];
            for (int a = 0; a < 3; ++a) {
                r[a] = x[a] - c[a];
                r2 += r[a] * r[a];
            }
            const double s2 = r2 + eps * eps;
            for (int a = 0; a < 3; ++a) A[a] += m * r[a] / (s2 * sqrt(s2));
            m_all += m;
            if (is_cell) {
                double d2 = 0.0;
                for (int a = 0; a < 3; ++a) {
                    double d = 0.0;
                    if (blo[a] - x[a] > d) d = blo[a] - x[a];
                    if (x[a] - bhi[a] > d) d = x[a] - bhi[a];
                    d2 += d * d;
                }
                const double d = sqrt(d2);
                if (d / cn->side < min_ratio) min_ratio = d / cn->side;
                m_cells += m;
                const double dd = d > 1e-300 ? d : 1e-300;
                T += cn->b2 * cn->bmax / (dd * dd * dd * dd * dd);
            }
        }
        const int64_t len = ent.n_cell + ent.n_part;
        double A_abs = sqrt(A[0] * A[0] + A[1] * A[1] + A[2] * A[2]);
        if (A_abs < 1e-300) A_abs = 1e-300;
        double tr = T / A_abs;
        if (tr < 1e-12) tr = 1e-12;
        g_key[g] = key;
        feat[5 * g + 0] = log2((double)(len > 1 ? len : 1));
        feat[5 * g + 1] = log10(min_ratio > 1e-3 ? min_ratio : 1e-3);
        feat[5 * g + 2] = log10(h / eps);
        feat[5 * g + 3] = m_all > 0.0 ? m_cells / m_all : 0.0;
        feat[5 * g + 4] = log10(tr);
        free((void*)ent.cell);
        free(ent.part);
    }
    return err ? -2 : 0;
}

/* ------------------------------------------------------------------------- */
/* SPH sums through the tree (Section II, Bounding Radius for SPH).          */
/* ------------------------------------------------------------------------- */

/* r_SPH = max over the cell's particles of |com - x_j| + h_j (Eq. SPH_RAD). */
static void set_rsph(const OracleTree* t, Node* c, const double* h)
{
    double r = 0.0;
    for (int64_t k = c->begin; k < c->end; ++k) {
        int64_t j = t->idx[k];
        double dx = c->com[0] - t->pos[3 * j], dy = c->com[1] - t->pos[3 * j + 1], dz = c->com[2] - t->pos[3 * j + 2];
        double v = sqrt(dx * dx + dy * dy + dz * dz) + h[j];
        if (v > r) r = v;
    }
    c->rsph = r;
    for (int k = 0; k < c->n_child; ++k) set_rsph(t, c->child[k], h);
}

/* The SPH walk: a cell whose sphere (centre of mass, r_SPH) lies farther
   than r_SPH from the group box holds no neighbour of any group particle and
   is skipped; other cells open; leaves give their particles. */
static int sph_walk(const OracleTree* t, const Node* c, const double blo[3], const double bhi[3], Entries* e)
{
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        double d = 0.0;
        if (blo[a] - c->com[a] > d) d = blo[a] - c->com[a];
        if (c->com[a] - bhi[a] > d) d = c->com[a] - bhi[a];
        d2 += d * d;
    }
    if (sqrt(d2) > c->rsph) return 0;
    if (c->n_child == 0) {
        for (int64_t k = c->begin; k < c->end; ++k)
            if (push_part(e, t->idx[k])) return -1;
        return 0;
    }
    for (int k = 0; k < c->n_child; ++k)
        if (sph_walk(t, c->child[k], blo, bhi, e)) return -1;
    return 0;
}

/* Density of every particle through the tree's groups (caller order, rho
   [n]); per-group statistics g_key (lowest particle index), g_npart
   (particle entries); *pairs = sum over groups of count * entries. */
int oracle_tree_sph_density(void* handle, const double* h, double* rho, int64_t* g_key, int64_t* g_npart,
                            int64_t* pairs)
{
    OracleTree* t = (OracleTree*)handle;
    if (!t) return -1;
    for (int64_t j = 0; j < t->n; ++j)
        if (!(h[j] > 0.0)) return -1;
    set_rsph(t, t->root, h);
    int64_t total = 0;
    int err = 0;
    int64_t g;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total) reduction(| : err)
    for (g = 0; g < t->n_groups; ++g) {
        int64_t b = t->grp_begin[g], e_ = t->grp_end[g];
        double blo[3], bhi[3];
        int64_t key = t->idx[b];
        for (int a = 0; a < 3; ++a) blo[a] = bhi[a] = t->pos[3 * t->idx[b] + a];
        for (int64_t k = b; k < e_; ++k) {
            int64_t i = t->idx[k];
            if (i < key) key = i;
            for (int a = 0; a < 3; ++a) {
                if (t->pos[3 * i + a] < blo[a]) blo[a] = t->pos[3 * i + a];
                if (t->pos[3 * i + a] > bhi[a]) bhi[a] = t->pos[3 * i + a];
            }
        }
        Entries ent;
        memset(&ent, 0, sizeof(ent));
        if (sph_walk(t, t->root, blo, bhi, &ent)) {
            err |= 1;
            free(ent.part);
            continue;
        }
        if (g_key) g_key[g] = key;
        if (g_npart) g_npart[g] = ent.n_part;
        total += (e_ - b) * ent.n_part;
        for (int64_t k = b; k < e_; ++k) {
            int64_t i = t->idx[k];
            double s = 0.0;
            for (int64_t q = 0; q < ent.n_part; ++q) {
                int64_t j = ent.part[q];
                double dx = t->pos[3 * j] - t->pos[3 * i], dy = t->pos[3 * j + 1] - t->pos[3 * i + 1],
                       dz = t->pos[3 * j + 2] - t->pos[3 * i + 2];
                s += t->mass[j] * sph_w(sqrt(dx * dx + dy * dy + dz * dz), h[j]);
            }
            rho[i] = s;
        }
        free(ent.part);
    }
    if (pairs) *pairs = total;
    return err ? -2 : 0;
}
