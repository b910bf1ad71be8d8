/*
 * octgrav_oracle.c -- plain, slow FP64 CPU reference of the grouped Barnes-Hut
 * force calculation of Gaburov, Bedorf & Portegies Zwart (2010),
 * "Gravitational tree-code on graphics processing units: implementation in
 * CUDA".
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this file. It shares no code, header, table or helper
 * with the CUDA path; both implement the same definitions independently.
 *
 * What it computes, step by step in the paper's order:
 *   O1  direct Plummer-softened summation (the exact result the tree
 *       approximates; the paper's accuracy reference, Sec. 3.1);
 *   O2  octree: a cube around all particles split recursively into octants
 *       until a cell holds no more than N_leaf particles (Sec. 2.1, Fig. 1);
 *       groups are the largest cells holding no more than N_group particles
 *       (Sec. 2.1, Sec. 2.2);
 *   O3  per cell: tight bounding box, boundary cube (side = longest side of
 *       the box, same centre; Fig. 1), mass, centre of mass and second
 *       moments (Sec. 2.1), each summed directly over the cell's members;
 *   O4  opening test of a cell against a group (Sec. 2.2, Listing 2),
 *       evaluated in FP32 round-to-nearest without contraction so that a
 *       second implementation can reproduce every decision bit for bit;
 *   O5  per group, a walk from the root that sorts each child of an opened
 *       node into the stack (opened node), the leaf list (opened leaf) or the
 *       cell list (accepted cell) (Sec. 2.2, Listings 1 and 2);
 *   O6  accelerations and potentials: particle-cell interactions as the
 *       second-order Taylor expansion of the Plummer kernel about the cell's
 *       centre of mass (monopole + quadrupole), particle-particle interactions
 *       with every member of each leaf in the leaf list except the particle
 *       itself (Sec. 2.3, Listings 3 and 4).
 *
 * Readings of points the paper leaves open (each one is listed in the design
 * notes):
 *   - root cube: centre = centre of the bounding box of all particles, side =
 *     longest box side * (1 + 2^-20) (1.0 if all particles coincide);
 *   - octant membership: u = (x - lo) / side in FP64, q = floor(u * 2^D)
 *     clamped to [0, 2^D - 1], D = max depth = 21; the child of a depth-L
 *     cell is chosen by bit (D-1-L) of q on each axis (x is octant bit 0);
 *   - a cell is a leaf when it holds <= N_leaf particles or sits at depth D;
 *   - a cell's key is (1 << 3L) | (octant path), independent of storage order;
 *   - opening test: l = boundary cube side = 2h, d = distance between the
 *     group's tight box and the cell's boundary cube (0 when they overlap);
 *     the cell is opened iff l >= theta * d, evaluated as
 *     4*(h*h) >= fl32(theta^2) * ((dx*dx + dy*dy) + dz*dz) in FP32;
 *   - the root is always opened; a group whose cell is the root's leaf gets
 *     the root in its leaf list;
 *   - the self term (j == i) is left out of both acceleration and potential.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -fPIC -shared -pthread
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORA_MAX_DEPTH 21

/* ------------------------------------------------------------------------ */
/* O1: direct summation                                                      */
/* ------------------------------------------------------------------------ */

/* a_i = G sum_{j != i} m_j (x_j - x_i) / (|x_j - x_i|^2 + eps^2)^{3/2}
 * phi_i = -G sum_{j != i} m_j / (|x_j - x_i|^2 + eps^2)^{1/2}
 * Plummer softening; the paper's accuracy reference (Sec. 3.1) is plain
 * direct summation. */
static void direct_one(const double *pos, const double *mass, int64_t n, int64_t i,
                       double eps2, double G, double *a, double *p)
{
    double ax = 0, ay = 0, az = 0, phi = 0;
    const double xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
    for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        double dx = pos[3 * j] - xi, dy = pos[3 * j + 1] - yi, dz = pos[3 * j + 2] - zi;
        double r2 = dx * dx + dy * dy + dz * dz + eps2;
        if (r2 == 0.0) continue; /* coincident particles with eps = 0 */
        double rinv = 1.0 / sqrt(r2);
        double mr3 = mass[j] * rinv * rinv * rinv;
        ax += mr3 * dx; ay += mr3 * dy; az += mr3 * dz;
        phi -= mass[j] * rinv;
    }
    a[0] = G * ax; a[1] = G * ay; a[2] = G * az;
    *p = G * phi;
}

typedef struct {
    const double *pos, *mass; int64_t n;
    const int64_t *targets; int64_t nt;
    double eps2, G; double *acc, *pot;
    int64_t next; /* atomic work counter */
} direct_job;

static void *direct_worker(void *arg)
{
    direct_job *J = (direct_job *)arg;
    for (;;) {
        int64_t k = __atomic_fetch_add(&J->next, 1, __ATOMIC_RELAXED);
        if (k >= J->nt) break;
        int64_t i = J->targets ? J->targets[k] : k;
        direct_one(J->pos, J->mass, J->n, i, J->eps2, J->G, J->acc + 3 * k, J->pot + k);
    }
    return NULL;
}

static void run_threads(void *(*fn)(void *), void *job, int nthreads)
{
    if (nthreads <= 1) { fn(job); return; }
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    int started = 0;
    for (int t = 0; t < nthreads; ++t)
        if (pthread_create(&th[t], NULL, fn, job) == 0) ++started;
    if (started == 0) fn(job);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    free(th);
}

/* targets == NULL means all particles (nt must equal n). */
int ora_direct(const double *pos, const double *mass, int64_t n, const int64_t *targets,
               int64_t nt, double eps, double G, double *acc, double *pot, int nthreads)
{
    direct_job J = {pos, mass, n, targets, nt, eps * eps, G, acc, pot, 0};
    run_threads(direct_worker, &J, nthreads);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* O2 + O3: octree, cell properties, groups                                  */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t n;
    int n_leaf, n_group, max_depth;
    const double *pos, *mass;   /* caller-owned, must outlive the tree */
    double lo[3], side;          /* quantisation frame (root cube) */
    uint64_t *q;                 /* 3 per particle */
    int64_t *idx;                /* particle indices, partitioned cell by cell */
    int64_t *tmp;
    /* cells in creation (depth-first pre-)order */
    int64_t n_cells, cap;
    uint64_t *key;
    int32_t *depth;
    int64_t *parent;
    int64_t *child;              /* 8 per cell, -1 = empty octant */
    int64_t *first, *count;      /* members: idx[first .. first+count) */
    int32_t *leaf;
    double *bmin, *bmax;         /* 3 per cell: tight bounding box */
    double *cube;                /* 4 per cell: boundary cube centre xyz, half side h */
    double *M, *com, *S;         /* mass; 3; 6 (xx, yy, zz, xy, xz, yz) */
    int64_t n_groups, gcap;
    int64_t *group;              /* cell index of each group, depth-first order */
} ora_tree;

static int grow_cells(ora_tree *T)
{
    int64_t nc = T->cap ? T->cap * 2 : 1024;
#define GROW(f, type, k) do { void *p_ = realloc(T->f, sizeof(type) * (size_t)(k) * (size_t)nc); \
        if (!p_) return -1; T->f = (type *)p_; } while (0)
    GROW(key, uint64_t, 1); GROW(depth, int32_t, 1); GROW(parent, int64_t, 1);
    GROW(child, int64_t, 8); GROW(first, int64_t, 1); GROW(count, int64_t, 1);
    GROW(leaf, int32_t, 1); GROW(bmin, double, 3); GROW(bmax, double, 3);
    GROW(cube, double, 4); GROW(M, double, 1); GROW(com, double, 3); GROW(S, double, 6);
#undef GROW
    T->cap = nc;
    return 0;
}

/* Cell properties summed directly over the members (O3). */
static void cell_props(ora_tree *T, int64_t c)
{
    const int64_t f = T->first[c], k = T->count[c];
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    double M = 0, cx = 0, cy = 0, cz = 0;
    for (int64_t a = f; a < f + k; ++a) {
        int64_t i = T->idx[a];
        const double *x = T->pos + 3 * i;
        for (int d = 0; d < 3; ++d) { if (x[d] < mn[d]) mn[d] = x[d]; if (x[d] > mx[d]) mx[d] = x[d]; }
        M += T->mass[i];
        cx += T->mass[i] * x[0]; cy += T->mass[i] * x[1]; cz += T->mass[i] * x[2];
    }
    double *cu = T->cube + 4 * c;
    for (int d = 0; d < 3; ++d) {
        T->bmin[3 * c + d] = mn[d]; T->bmax[3 * c + d] = mx[d];
        cu[d] = (mn[d] + mx[d]) * 0.5;
    }
    double ext = mx[0] - mn[0];
    if (mx[1] - mn[1] > ext) ext = mx[1] - mn[1];
    if (mx[2] - mn[2] > ext) ext = mx[2] - mn[2];
    cu[3] = 0.5 * ext;
    T->M[c] = M;
    double *cm = T->com + 3 * c;
    if (M > 0) { cm[0] = cx / M; cm[1] = cy / M; cm[2] = cz / M; }
    else { cm[0] = cu[0]; cm[1] = cu[1]; cm[2] = cu[2]; }
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t a = f; a < f + k; ++a) {
        int64_t i = T->idx[a];
        const double *x = T->pos + 3 * i;
        double y0 = x[0] - cm[0], y1 = x[1] - cm[1], y2 = x[2] - cm[2], m = T->mass[i];
        s[0] += m * y0 * y0; s[1] += m * y1 * y1; s[2] += m * y2 * y2;
        s[3] += m * y0 * y1; s[4] += m * y0 * y2; s[5] += m * y1 * y2;
    }
    memcpy(T->S + 6 * c, s, sizeof s);
}

/* Recursive subdivision (O2). Returns the new cell index or -1 on OOM. */
static int64_t build_cell(ora_tree *T, int depth, uint64_t key, int64_t first, int64_t count,
                          int64_t parent)
{
    if (T->n_cells == T->cap && grow_cells(T)) return -1;
    const int64_t c = T->n_cells++;
    T->key[c] = key; T->depth[c] = depth; T->parent[c] = parent;
    T->first[c] = first; T->count[c] = count;
    for (int o = 0; o < 8; ++o) T->child[8 * c + o] = -1;
    cell_props(T, c);
    if (count <= T->n_leaf || depth >= T->max_depth) { T->leaf[c] = 1; return c; }
    T->leaf[c] = 0;
    /* stable partition of the members into the 8 octants */
    const int bit = T->max_depth - 1 - depth;
    int64_t cnt[8] = {0}, off[8];
    for (int64_t a = first; a < first + count; ++a) {
        const uint64_t *q = T->q + 3 * T->idx[a];
        int o = (int)(((q[0] >> bit) & 1) | (((q[1] >> bit) & 1) << 1) | (((q[2] >> bit) & 1) << 2));
        cnt[o]++;
    }
    off[0] = first;
    for (int o = 1; o < 8; ++o) off[o] = off[o - 1] + cnt[o - 1];
    int64_t pos[8];
    memcpy(pos, off, sizeof pos);
    for (int64_t a = first; a < first + count; ++a) {
        const uint64_t *q = T->q + 3 * T->idx[a];
        int o = (int)(((q[0] >> bit) & 1) | (((q[1] >> bit) & 1) << 1) | (((q[2] >> bit) & 1) << 2));
        T->tmp[pos[o]++] = T->idx[a];
    }
    memcpy(T->idx + first, T->tmp + first, sizeof(int64_t) * (size_t)count);
    for (int o = 0; o < 8; ++o) {
        if (!cnt[o]) continue;
        int64_t ch = build_cell(T, depth + 1, (key << 3) | (uint64_t)o, off[o], cnt[o], c);
        if (ch < 0) return -1;
        T->child[8 * c + o] = ch;
    }
    return c;
}

/* Groups: descend from the root; a cell that is a leaf or holds no more than
 * N_group particles is a group, otherwise its children are examined. */
static int collect_groups(ora_tree *T, int64_t c)
{
    if (T->leaf[c] || T->count[c] <= T->n_group) {
        if (T->n_groups == T->gcap) {
            int64_t nc = T->gcap ? 2 * T->gcap : 1024;
            int64_t *p = (int64_t *)realloc(T->group, sizeof(int64_t) * (size_t)nc);
            if (!p) return -1;
            T->group = p; T->gcap = nc;
        }
        T->group[T->n_groups++] = c;
        return 0;
    }
    for (int o = 0; o < 8; ++o)
        if (T->child[8 * c + o] >= 0 && collect_groups(T, T->child[8 * c + o])) return -1;
    return 0;
}

void ora_tree_free(ora_tree *T)
{
    if (!T) return;
    free(T->q); free(T->idx); free(T->tmp);
    free(T->key); free(T->depth); free(T->parent); free(T->child); free(T->first);
    free(T->count); free(T->leaf); free(T->bmin); free(T->bmax); free(T->cube);
    free(T->M); free(T->com); free(T->S); free(T->group);
    free(T);
}

/* The caller keeps pos and mass alive for the lifetime of the tree. */
ora_tree *ora_tree_build(const double *pos, const double *mass, int64_t n, int n_leaf,
                         int n_group, int max_depth)
{
    if (n <= 0 || n_leaf < 1 || n_group < n_leaf || max_depth < 1 || max_depth > ORA_MAX_DEPTH)
        return NULL;
    ora_tree *T = (ora_tree *)calloc(1, sizeof(ora_tree));
    if (!T) return NULL;
    T->n = n; T->n_leaf = n_leaf; T->n_group = n_group; T->max_depth = max_depth;
    T->pos = pos; T->mass = mass;
    /* root cube */
    double mn[3], mx[3];
    for (int d = 0; d < 3; ++d) { mn[d] = pos[d]; mx[d] = pos[d]; }
    for (int64_t i = 1; i < n; ++i)
        for (int d = 0; d < 3; ++d) {
            if (pos[3 * i + d] < mn[d]) mn[d] = pos[3 * i + d];
            if (pos[3 * i + d] > mx[d]) mx[d] = pos[3 * i + d];
        }
    double ext = mx[0] - mn[0];
    if (mx[1] - mn[1] > ext) ext = mx[1] - mn[1];
    if (mx[2] - mn[2] > ext) ext = mx[2] - mn[2];
    if (!(ext > 0)) ext = 1.0;
    T->side = ext * (1.0 + 1.0 / 1048576.0);
    for (int d = 0; d < 3; ++d) T->lo[d] = (mn[d] + mx[d]) * 0.5 - T->side * 0.5;
    /* quantised coordinates */
    T->q = (uint64_t *)malloc(sizeof(uint64_t) * 3 * (size_t)n);
    T->idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    T->tmp = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!T->q || !T->idx || !T->tmp) { ora_tree_free(T); return NULL; }
    const double scale = ldexp(1.0, max_depth);
    const uint64_t qmax = ((uint64_t)1 << max_depth) - 1;
    for (int64_t i = 0; i < n; ++i) {
        T->idx[i] = i;
        for (int d = 0; d < 3; ++d) {
            double u = (pos[3 * i + d] - T->lo[d]) / T->side;
            double v = floor(u * scale);
            uint64_t qq = v <= 0 ? 0 : (v >= (double)qmax ? qmax : (uint64_t)v);
            T->q[3 * i + d] = qq;
        }
    }
    if (build_cell(T, 0, 1, 0, n, -1) < 0 || collect_groups(T, 0)) { ora_tree_free(T); return NULL; }
    return T;
}

/* ---- accessors (copy out) ---- */
void ora_tree_info(const ora_tree *T, int64_t *out /* 6 */)
{
    int64_t leaves = 0;
    for (int64_t c = 0; c < T->n_cells; ++c) leaves += T->leaf[c];
    out[0] = T->n; out[1] = T->n_cells; out[2] = leaves; out[3] = T->n_groups;
    out[4] = T->max_depth; out[5] = 0;
    for (int64_t c = 0; c < T->n_cells; ++c) if (T->depth[c] > out[5]) out[5] = T->depth[c];
}

void ora_tree_frame(const ora_tree *T, double *lo_side /* 4 */)
{
    lo_side[0] = T->lo[0]; lo_side[1] = T->lo[1]; lo_side[2] = T->lo[2]; lo_side[3] = T->side;
}

void ora_tree_cells(const ora_tree *T, uint64_t *key, int32_t *depth, int64_t *parent,
                    int32_t *leaf, int64_t *first, int64_t *count, int64_t *child,
                    double *bmin, double *bmax, double *cube, double *M, double *com, double *S)
{
    const size_t nc = (size_t)T->n_cells;
    if (key) memcpy(key, T->key, 8 * nc);
    if (depth) memcpy(depth, T->depth, 4 * nc);
    if (parent) memcpy(parent, T->parent, 8 * nc);
    if (leaf) memcpy(leaf, T->leaf, 4 * nc);
    if (first) memcpy(first, T->first, 8 * nc);
    if (count) memcpy(count, T->count, 8 * nc);
    if (child) memcpy(child, T->child, 64 * nc);
    if (bmin) memcpy(bmin, T->bmin, 24 * nc);
    if (bmax) memcpy(bmax, T->bmax, 24 * nc);
    if (cube) memcpy(cube, T->cube, 32 * nc);
    if (M) memcpy(M, T->M, 8 * nc);
    if (com) memcpy(com, T->com, 24 * nc);
    if (S) memcpy(S, T->S, 48 * nc);
}

void ora_tree_members(const ora_tree *T, int64_t *idx /* n */)
{
    memcpy(idx, T->idx, sizeof(int64_t) * (size_t)T->n);
}

void ora_tree_groups(const ora_tree *T, int64_t *group /* n_groups */)
{
    memcpy(group, T->group, sizeof(int64_t) * (size_t)T->n_groups);
}

/* ------------------------------------------------------------------------ */
/* O4: opening test (FP32, round to nearest, no contraction)                 */
/* ------------------------------------------------------------------------ */

/* Distance between the group's tight box [gmin, gmax] and the cell's boundary
 * cube (centre c, half side h); the cell is opened iff its side 2h is at least
 * theta times that distance. Returns 1 = open, 0 = accept. */
static float gap2_f32(const float gmin[3], const float gmax[3], const float c[3], float h)
{
    float d[3];
    for (int k = 0; k < 3; ++k) {
        float below = gmin[k] - (c[k] + h); /* cube lies below the group box */
        float above = (c[k] - h) - gmax[k]; /* cube lies above the group box */
        float t = below > above ? below : above;
        d[k] = t > 0.0f ? t : 0.0f;
    }
    return (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
}

int ora_open_f32(const float gmin[3], const float gmax[3], const float c[3], float h,
                 float theta2)
{
    float d2 = gap2_f32(gmin, gmax, c, h);
    float lhs = 4.0f * (h * h);
    return lhs >= theta2 * d2;
}

/* Same test in FP64 (diagnostic only: counts decisions that FP32 flips). */
static int open_f64(const double *gmin, const double *gmax, const double *c, double h, double theta)
{
    double d2 = 0;
    for (int k = 0; k < 3; ++k) {
        double below = gmin[k] - (c[k] + h), above = (c[k] - h) - gmax[k];
        double t = below > above ? below : above;
        if (t > 0) d2 += t * t;
    }
    return 4.0 * h * h >= theta * theta * d2;
}

static int open_cell(const ora_tree *T, int64_t g, int64_t c, float theta2)
{
    const int64_t gc = T->group[g];
    float gmin[3], gmax[3], cc[3];
    for (int k = 0; k < 3; ++k) {
        gmin[k] = (float)T->bmin[3 * gc + k];
        gmax[k] = (float)T->bmax[3 * gc + k];
        cc[k] = (float)T->cube[4 * c + k];
    }
    return ora_open_f32(gmin, gmax, cc, (float)T->cube[4 * c + 3], theta2);
}

/* The squared box-to-cube distance exactly as the opening test sees it (FP32). */
static float cell_gap2_f32(const ora_tree *T, int64_t g, int64_t c)
{
    const int64_t gc = T->group[g];
    float gmin[3], gmax[3], cc[3];
    for (int k = 0; k < 3; ++k) {
        gmin[k] = (float)T->bmin[3 * gc + k];
        gmax[k] = (float)T->bmax[3 * gc + k];
        cc[k] = (float)T->cube[4 * c + k];
    }
    return gap2_f32(gmin, gmax, cc, (float)T->cube[4 * c + 3]);
}

/* ------------------------------------------------------------------------ */
/* O5: walk and list classification                                          */
/* ------------------------------------------------------------------------ */

typedef struct { int64_t *v; int64_t n, cap; } vec;

static int vpush(vec *a, int64_t x)
{
    if (a->n == a->cap) {
        int64_t nc = a->cap ? 2 * a->cap : 256;
        int64_t *p = (int64_t *)realloc(a->v, sizeof(int64_t) * (size_t)nc);
        if (!p) return -1;
        a->v = p; a->cap = nc;
    }
    a->v[a->n++] = x;
    return 0;
}

/* Walk for group g: the root is opened; every child of an opened node is
 * tested: opened node -> examined in turn, opened leaf -> leaf list, accepted
 * cell (node or leaf) -> cell list. Depth-first with an explicit stack.
 * flips (optional) counts children whose FP64 decision differs. */
static int walk_group(const ora_tree *T, int64_t g, float theta2, double theta,
                      vec *cells, vec *leaves, int64_t *flips)
{
    cells->n = 0; leaves->n = 0;
    if (T->leaf[0]) return vpush(leaves, 0);
    vec stack = {0, 0, 0};
    if (vpush(&stack, 0)) return -1;
    const int64_t gc = T->group[g];
    while (stack.n) {
        int64_t node = stack.v[--stack.n];
        for (int o = 0; o < 8; ++o) {
            int64_t ch = T->child[8 * node + o];
            if (ch < 0) continue;
            int op = open_cell(T, g, ch, theta2);
            if (flips && op != open_f64(T->bmin + 3 * gc, T->bmax + 3 * gc, T->cube + 4 * ch,
                                        T->cube[4 * ch + 3], theta)) ++*flips;
            int rc;
            if (op) rc = T->leaf[ch] ? vpush(leaves, ch) : vpush(&stack, ch);
            else rc = vpush(cells, ch);
            if (rc) { free(stack.v); return -1; }
        }
    }
    free(stack.v);
    return 0;
}

static float theta2_f32(double theta) { return (float)(theta * theta); }

/* Lists of one group as cell indices. Returns the total number of entries
 * needed; writes at most cap_c / cap_l entries. *n_c / *n_l get the sizes. */
int64_t ora_walk(const ora_tree *T, int64_t g, double theta, int64_t *cell_out, int64_t cap_c,
                 int64_t *n_c, int64_t *leaf_out, int64_t cap_l, int64_t *n_l)
{
    if (g < 0 || g >= T->n_groups) return -1;
    vec cells = {0, 0, 0}, leaves = {0, 0, 0};
    if (walk_group(T, g, theta2_f32(theta), theta, &cells, &leaves, NULL)) return -1;
    for (int64_t k = 0; k < cells.n && k < cap_c; ++k) cell_out[k] = cells.v[k];
    for (int64_t k = 0; k < leaves.n && k < cap_l; ++k) leaf_out[k] = leaves.v[k];
    *n_c = cells.n; *n_l = leaves.n;
    int64_t tot = cells.n + leaves.n;
    free(cells.v); free(leaves.v);
    return tot;
}

/* ------------------------------------------------------------------------ */
/* O6: evaluation                                                            */
/* ------------------------------------------------------------------------ */

/* Field of cell c at point x, second-order Taylor expansion of the Plummer
 * kernel about the centre of mass. With y = x - com, r^2 = |y|^2 + eps^2,
 * S = sum m (x_j - com)(x_j - com)^T:
 *   phi = -G [ M/r + (3/2) y.S.y / r^5 - (1/2) tr S / r^3 ]
 *   a   =  G [ -M y/r^3 + 3 S y / r^5 - (15/2) (y.S.y) y / r^7 + (3/2) tr S y / r^5 ] */
void ora_cell_field(const double *com, double M, const double *S, const double *x, double eps2,
                    double G, double *a, double *phi)
{
    double y0 = x[0] - com[0], y1 = x[1] - com[1], y2 = x[2] - com[2];
    double r2 = y0 * y0 + y1 * y1 + y2 * y2 + eps2;
    double r = sqrt(r2);
    double r3 = r2 * r, r5 = r3 * r2, r7 = r5 * r2;
    double Sy0 = S[0] * y0 + S[3] * y1 + S[4] * y2;
    double Sy1 = S[3] * y0 + S[1] * y1 + S[5] * y2;
    double Sy2 = S[4] * y0 + S[5] * y1 + S[2] * y2;
    double ySy = y0 * Sy0 + y1 * Sy1 + y2 * Sy2;
    double trS = S[0] + S[1] + S[2];
    double cy = -M / r3 - 7.5 * ySy / r7 + 1.5 * trS / r5;
    a[0] = G * (cy * y0 + 3.0 * Sy0 / r5);
    a[1] = G * (cy * y1 + 3.0 * Sy1 / r5);
    a[2] = G * (cy * y2 + 3.0 * Sy2 / r5);
    *phi = -G * (M / r + 1.5 * ySy / r5 - 0.5 * trS / r3);
}

static int cmp_key_idx(const void *a, const void *b, void *keys)
{
    const uint64_t *K = (const uint64_t *)keys;
    uint64_t ka = K[*(const int64_t *)a], kb = K[*(const int64_t *)b];
    return ka < kb ? -1 : ka > kb;
}

/* qsort_r is not portable C; a small insertion/merge sort keeps this plain. */
static void sort_by_key(int64_t *v, int64_t n, const uint64_t *keys, int64_t *tmp)
{
    if (n < 2) return;
    if (n <= 16) {
        for (int64_t i = 1; i < n; ++i) {
            int64_t x = v[i], j = i;
            while (j > 0 && cmp_key_idx(&v[j - 1], &x, (void *)keys) > 0) { v[j] = v[j - 1]; --j; }
            v[j] = x;
        }
        return;
    }
    int64_t h = n / 2;
    sort_by_key(v, h, keys, tmp);
    sort_by_key(v + h, n - h, keys, tmp);
    int64_t i = 0, j = h, k = 0;
    while (i < h && j < n) tmp[k++] = (cmp_key_idx(&v[j], &v[i], (void *)keys) < 0) ? v[j++] : v[i++];
    while (i < h) tmp[k++] = v[i++];
    while (j < n) tmp[k++] = v[j++];
    memcpy(v, tmp, sizeof(int64_t) * (size_t)n);
}

typedef struct {
    const ora_tree *T;
    double eps2, G, theta; float theta2;
    const int64_t *groups; int64_t ng;   /* NULL = all groups */
    double *acc, *pot;                    /* input order, n entries */
    int64_t *npp, *npc;                   /* per particle, input order (optional) */
    int64_t next;
    int64_t flips;
    int err;
} forces_job;

static void *forces_worker(void *arg)
{
    forces_job *J = (forces_job *)arg;
    const ora_tree *T = J->T;
    vec cells = {0, 0, 0}, leaves = {0, 0, 0};
    int64_t *tmp = NULL; int64_t tcap = 0;
    int64_t flips = 0;
    for (;;) {
        int64_t k = __atomic_fetch_add(&J->next, 1, __ATOMIC_RELAXED);
        if (k >= J->ng) break;
        int64_t g = J->groups ? J->groups[k] : k;
        if (walk_group(T, g, J->theta2, J->theta, &cells, &leaves, &flips)) { J->err = -1; break; }
        int64_t need = cells.n > leaves.n ? cells.n : leaves.n;
        if (need > tcap) { free(tmp); tcap = need; tmp = (int64_t *)malloc(sizeof(int64_t) * (size_t)tcap); }
        sort_by_key(cells.v, cells.n, T->key, tmp);
        sort_by_key(leaves.v, leaves.n, T->key, tmp);
        const int64_t gc = T->group[g];
        int64_t pp_src = 0;
        for (int64_t l = 0; l < leaves.n; ++l) pp_src += T->count[leaves.v[l]];
        for (int64_t a = T->first[gc]; a < T->first[gc] + T->count[gc]; ++a) {
            const int64_t i = T->idx[a];
            const double *xi = T->pos + 3 * i;
            double ax = 0, ay = 0, az = 0, phi = 0;
            for (int64_t e = 0; e < cells.n; ++e) {
                const int64_t c = cells.v[e];
                double ac[3], pc;
                ora_cell_field(T->com + 3 * c, T->M[c], T->S + 6 * c, xi, J->eps2, 1.0, ac, &pc);
                ax += ac[0]; ay += ac[1]; az += ac[2]; phi += pc;
            }
            for (int64_t e = 0; e < leaves.n; ++e) {
                const int64_t c = leaves.v[e];
                for (int64_t b = T->first[c]; b < T->first[c] + T->count[c]; ++b) {
                    const int64_t j = T->idx[b];
                    if (j == i) continue;
                    const double *xj = T->pos + 3 * j;
                    double dx = xj[0] - xi[0], dy = xj[1] - xi[1], dz = xj[2] - xi[2];
                    double r2 = dx * dx + dy * dy + dz * dz + J->eps2;
                    if (r2 == 0.0) continue;
                    double rinv = 1.0 / sqrt(r2);
                    double mr3 = T->mass[j] * rinv * rinv * rinv;
                    ax += mr3 * dx; ay += mr3 * dy; az += mr3 * dz;
                    phi -= T->mass[j] * rinv;
                }
            }
            J->acc[3 * i] = J->G * ax; J->acc[3 * i + 1] = J->G * ay; J->acc[3 * i + 2] = J->G * az;
            J->pot[i] = J->G * phi;
            if (J->npp) J->npp[i] = pp_src - 1;
            if (J->npc) J->npc[i] = cells.n;
        }
    }
    __atomic_fetch_add(&J->flips, flips, __ATOMIC_RELAXED);
    free(cells.v); free(leaves.v); free(tmp);
    return NULL;
}

/* Tree forces for the particles of the listed groups (all groups when groups
 * == NULL). acc/pot/npp/npc are indexed by input particle index; entries of
 * particles outside the listed groups are left untouched. Returns the number
 * of opening decisions whose FP64 evaluation differs from FP32, or -1. */
int64_t ora_forces(const ora_tree *T, double eps, double theta, double G, const int64_t *groups,
                   int64_t ng, double *acc, double *pot, int64_t *npp, int64_t *npc, int nthreads)
{
    forces_job J;
    memset(&J, 0, sizeof J);
    J.T = T; J.eps2 = eps * eps; J.G = G; J.theta = theta; J.theta2 = theta2_f32(theta);
    J.groups = groups; J.ng = groups ? ng : T->n_groups;
    J.acc = acc; J.pot = pot; J.npp = npp; J.npc = npc;
    run_threads(forces_worker, &J, nthreads);
    return J.err ? -1 : J.flips;
}

/* ------------------------------------------------------------------------ */
/* O8: learned opening criterion -- features, error labels, MLP walk        */
/* ------------------------------------------------------------------------ */

#define ORA_NF 12
#define ORA_NH 64

/* Box-to-cube distance in FP64 (the quantity the opening test compares). */
static double box_cube_dist(const double *gmin, const double *gmax, const double *cube)
{
    double d2 = 0, h = cube[3];
    for (int k = 0; k < 3; ++k) {
        double below = gmin[k] - (cube[k] + h), above = (cube[k] - h) - gmax[k];
        double t = below > above ? below : above;
        if (t > 0) d2 += t * t;
    }
    return sqrt(d2);
}

static double lg2(double x) { return log2(x > 1e-30 ? x : 1e-30); }

/* The 12 inputs of the learned criterion for group g and cell c (h > 0, d > 0):
 *  0 log2 l, 1 log2 d, 2 log2 |com_c - C_g|, 3 l/d, 4 log2 M_c,
 *  5 |S_c|_F / (M_c l^2), 6 log2 count_c, 7..9 group half extents / l,
 *  10 count_g / N_group, 11 log2 |C_g - com_root|,
 * with l = 2h the side of the cell's boundary cube, d the box-to-cube distance,
 * C_g the centre of the group's boundary cube. */
void ora_mlp_features(const ora_tree *T, int64_t g, int64_t c, double *f)
{
    const int64_t gc = T->group[g];
    const double *cu = T->cube + 4 * c, *C = T->cube + 4 * gc, *cm = T->com + 3 * c, *S = T->S + 6 * c;
    const double *rc = T->com; /* root centre of mass */
    const double l = 2.0 * cu[3];
    const double d = box_cube_dist(T->bmin + 3 * gc, T->bmax + 3 * gc, cu);
    double r2 = 0, o2 = 0;
    for (int k = 0; k < 3; ++k) { r2 += (cm[k] - C[k]) * (cm[k] - C[k]); o2 += (C[k] - rc[k]) * (C[k] - rc[k]); }
    const double sf = sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2] + 2.0 * (S[3] * S[3] + S[4] * S[4] + S[5] * S[5]));
    const double M = T->M[c];
    f[0] = lg2(l);
    f[1] = lg2(d);
    f[2] = lg2(sqrt(r2));
    f[3] = l / d;
    f[4] = lg2(M);
    f[5] = M > 0 ? sf / (M * l * l) : 0.0;
    f[6] = lg2((double)T->count[c]);
    for (int k = 0; k < 3; ++k) f[7 + k] = 0.5 * (T->bmax[3 * gc + k] - T->bmin[3 * gc + k]) / l;
    f[10] = (double)T->count[gc] / (double)T->n_group;
    f[11] = lg2(sqrt(o2));
}

/* Error label of accepting cell c for group g: the largest, over the group's
 * particles i, of |a_multipole(c, i) - a_direct(members of c, i)| / |a_ref(i)|,
 * a_ref the particle's total acceleration (input order, 3 per particle). The
 * direct part follows O1: the self term and coincident pairs at eps = 0
 * (r^2 = 0) are left out. */
static double mlp_label(const ora_tree *T, int64_t g, int64_t c, double eps2, const double *aref)
{
    const int64_t gc = T->group[g];
    double emax = 0;
    for (int64_t a = T->first[gc]; a < T->first[gc] + T->count[gc]; ++a) {
        const int64_t i = T->idx[a];
        const double *xi = T->pos + 3 * i;
        double am[3], pm;
        ora_cell_field(T->com + 3 * c, T->M[c], T->S + 6 * c, xi, eps2, 1.0, am, &pm);
        double ad[3] = {0, 0, 0};
        for (int64_t b = T->first[c]; b < T->first[c] + T->count[c]; ++b) {
            const int64_t j = T->idx[b];
            if (j == i) continue;
            const double *xj = T->pos + 3 * j;
            double dx = xj[0] - xi[0], dy = xj[1] - xi[1], dz = xj[2] - xi[2];
            double r2 = dx * dx + dy * dy + dz * dz + eps2;
            if (r2 == 0.0) continue;
            double rinv = 1.0 / sqrt(r2);
            double mr3 = T->mass[j] * rinv * rinv * rinv;
            ad[0] += mr3 * dx; ad[1] += mr3 * dy; ad[2] += mr3 * dz;
        }
        const double *ar = aref + 3 * i;
        double ea = sqrt((am[0] - ad[0]) * (am[0] - ad[0]) + (am[1] - ad[1]) * (am[1] - ad[1]) + (am[2] - ad[2]) * (am[2] - ad[2]));
        double na = sqrt(ar[0] * ar[0] + ar[1] * ar[1] + ar[2] * ar[2]);
        double e = na > 0 ? ea / na : 0;
        if (e > emax) emax = e;
    }
    return emax;
}

/* Training samples: for each listed group, every child tested by a walk with
 * opening parameter theta_walk whose cube has h > 0 and lies at d > 0 from the
 * group box yields (features, label, group, cell). h and d are taken as the
 * FP32 opening test sees them (the only pairs the criterion can be asked
 * about). Returns the number of samples (at most cap are written). */
typedef struct {
    const ora_tree *T; const int64_t *groups; int64_t ng; double theta, eps2; const double *aref;
    double *feat, *label; int64_t *pair; int64_t cap; int64_t *offs; int pass; int64_t next;
} samp_job;

static void *samp_worker(void *arg)
{
    samp_job *J = (samp_job *)arg;
    const ora_tree *T = J->T;
    const float theta2 = (float)(J->theta * J->theta);
    vec stack = {0, 0, 0};
    for (;;) {
        int64_t k = __atomic_fetch_add(&J->next, 1, __ATOMIC_RELAXED);
        if (k >= J->ng) break;
        const int64_t g = J->groups[k];
        int64_t cnt = 0, base = J->pass ? J->offs[k] : 0;
        stack.n = 0;
        if (!T->leaf[0]) vpush(&stack, 0);
        while (stack.n) {
            int64_t node = stack.v[--stack.n];
            for (int o = 0; o < 8; ++o) {
                int64_t ch = T->child[8 * node + o];
                if (ch < 0) continue;
                int op = open_cell(T, g, ch, theta2);
                if ((float)T->cube[4 * ch + 3] > 0.0f && cell_gap2_f32(T, g, ch) > 0.0f) {
                    if (J->pass) {
                        int64_t s = base + cnt;
                        if (s < J->cap) {
                            ora_mlp_features(T, g, ch, J->feat + ORA_NF * s);
                            J->label[s] = mlp_label(T, g, ch, J->eps2, J->aref);
                            J->pair[2 * s] = g; J->pair[2 * s + 1] = ch;
                        }
                    }
                    ++cnt;
                }
                if (op && !T->leaf[ch]) vpush(&stack, ch);
            }
        }
        if (!J->pass) J->offs[k] = cnt;
    }
    free(stack.v);
    return NULL;
}

int64_t ora_mlp_samples(const ora_tree *T, const int64_t *groups, int64_t ng, double theta_walk, double eps,
                        const double *aref, double *feat, double *label, int64_t *pair, int64_t cap, int nthreads)
{
    int64_t *offs = (int64_t *)calloc((size_t)ng + 1, sizeof(int64_t));
    samp_job J = {T, groups, ng, theta_walk, eps * eps, aref, feat, label, pair, cap, offs, 0, 0};
    run_threads(samp_worker, &J, nthreads);
    int64_t tot = 0;
    for (int64_t k = 0; k < ng; ++k) { int64_t c = offs[k]; offs[k] = tot; tot += c; }
    if (feat && label && pair && cap > 0) {
        J.pass = 1; J.next = 0;
        run_threads(samp_worker, &J, nthreads);
    }
    free(offs);
    return tot;
}

/* FP64 forward pass of the 12 -> 64 -> 64 -> 1 ReLU network. Layout of w:
 * W1[64][12], b1[64], W2[64][64], b2[64], w3[64], b3 (5057 values). */
double ora_mlp_forward(const double *w, const double *x)
{
    const double *W1 = w, *b1 = w + ORA_NH * ORA_NF, *W2 = b1 + ORA_NH, *b2 = W2 + ORA_NH * ORA_NH;
    const double *w3 = b2 + ORA_NH, *b3 = w3 + ORA_NH;
    double h1[ORA_NH], y = *b3;
    for (int j = 0; j < ORA_NH; ++j) {
        double s = b1[j];
        for (int i = 0; i < ORA_NF; ++i) s += W1[j * ORA_NF + i] * x[i];
        h1[j] = s > 0 ? s : 0;
    }
    for (int j = 0; j < ORA_NH; ++j) {
        double s = b2[j];
        for (int i = 0; i < ORA_NH; ++i) s += W2[j * ORA_NH + i] * h1[i];
        y += w3[j] * (s > 0 ? s : 0);
    }
    return y;
}

/* Round to the nearest BF16 value (8 significant bits, ties to even) by way of
 * FP32, as a tensor core's BF16 operand is made from an FP32 value. */
static double bf16_round(double v)
{
    float f = (float)v;
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) != 0x7f800000u) { /* finite: round the low 16 bits away */
        u += 0x7fffu + ((u >> 16) & 1u);
        u &= 0xffff0000u;
    }
    memcpy(&f, &u, 4);
    return (double)f;
}

/* The network with BF16 operands, the precision of a tensor-core evaluation
 * with BF16 weights: the inputs and the first hidden layer are rounded to
 * BF16 before they are multiplied (the weights w must already be BF16
 * values); sums, biases, the second hidden layer and the output stay exact
 * up to FP64. */
double ora_mlp_forward_bf16(const double *w, const double *x)
{
    const double *W1 = w, *b1 = w + ORA_NH * ORA_NF, *W2 = b1 + ORA_NH, *b2 = W2 + ORA_NH * ORA_NH;
    const double *w3 = b2 + ORA_NH, *b3 = w3 + ORA_NH;
    double xr[ORA_NF], h1[ORA_NH], y = *b3;
    for (int i = 0; i < ORA_NF; ++i) xr[i] = bf16_round(x[i]);
    for (int j = 0; j < ORA_NH; ++j) {
        double s = b1[j];
        for (int i = 0; i < ORA_NF; ++i) s += W1[j * ORA_NF + i] * xr[i];
        h1[j] = bf16_round(s > 0 ? s : 0);
    }
    for (int j = 0; j < ORA_NH; ++j) {
        double s = b2[j];
        for (int i = 0; i < ORA_NH; ++i) s += W2[j * ORA_NH + i] * h1[i];
        y += w3[j] * (s > 0 ? s : 0);
    }
    return y;
}

/* The learned criterion's decision for group g and child c (1 = open):
 * the FP32 opening test with theta_hi opens -> open; with theta_lo accepts ->
 * accept; otherwise (between the two) a cell with h = 0 is accepted (its
 * monopole is exact), a cell whose standardised features leave [fmin, fmax]
 * uses the FP32 test with theta_fb, and any other is accepted iff the network
 * predicts log10 error < tau (a prediction equal to tau opens).
 * Standardisation: x = (f - mu) / sigma. */
typedef struct {
    const double *w, *mu, *sigma, *fmin, *fmax; double tau, theta_lo, theta_hi, theta_fb;
    int bf16; /* 1: the network with BF16 operands (ora_mlp_forward_bf16) */
} mlp_rule;

/* Which rule decided a pair (ora_mlp_decide's *branch). */
enum { ORA_BR_HI_OPEN = 0, ORA_BR_LO_ACCEPT = 1, ORA_BR_POINT = 2, ORA_BR_FALLBACK = 3, ORA_BR_NETWORK = 4 };

static int mlp_open(const ora_tree *T, int64_t g, int64_t c, const mlp_rule *R, int *branch, double *y)
{
    *y = 0.0;
    if (open_cell(T, g, c, (float)(R->theta_hi * R->theta_hi))) { *branch = ORA_BR_HI_OPEN; return 1; }
    if (!open_cell(T, g, c, (float)(R->theta_lo * R->theta_lo))) { *branch = ORA_BR_LO_ACCEPT; return 0; }
    if ((float)T->cube[4 * c + 3] == 0.0f) { *branch = ORA_BR_POINT; return 0; }
    double f[ORA_NF], x[ORA_NF];
    ora_mlp_features(T, g, c, f);
    for (int i = 0; i < ORA_NF; ++i) {
        x[i] = (f[i] - R->mu[i]) / R->sigma[i];
        if (!(x[i] >= R->fmin[i] && x[i] <= R->fmax[i])) {
            *branch = ORA_BR_FALLBACK;
            return open_cell(T, g, c, (float)(R->theta_fb * R->theta_fb));
        }
    }
    *branch = ORA_BR_NETWORK;
    *y = R->bf16 ? ora_mlp_forward_bf16(R->w, x) : ora_mlp_forward(R->w, x);
    return !(*y < R->tau);
}

/* One decision of the learned criterion, exported for pair-by-pair checks:
 * returns 1 (open) or 0 (accept), or -1 for a bad group/cell index; *branch
 * receives the rule that decided (0 theta_hi opens, 1 theta_lo accepts,
 * 2 point cell h = 0, 3 out of the training range: theta_fb test, 4 network)
 * and *y the network's prediction (branch 4 only, else 0); bf16 = 1 evaluates
 * the network with BF16 operands (ora_mlp_forward_bf16). */
int ora_mlp_decide(const ora_tree *T, int64_t g, int64_t c, const double *w, const double *mu,
                   const double *sigma, const double *fmin, const double *fmax, double tau, double theta_lo,
                   double theta_hi, double theta_fb, int bf16, int *branch, double *y)
{
    if (g < 0 || g >= T->n_groups || c < 0 || c >= T->n_cells) return -1;
    mlp_rule R = {w, mu, sigma, fmin, fmax, tau, theta_lo, theta_hi, theta_fb, bf16};
    return mlp_open(T, g, c, &R, branch, y);
}

/* ora_mlp_decide for n pairs (groups[k], cells[k]): open[k], branch[k], y[k];
 * feat (n x 12, may be NULL) receives each pair's inputs where the rule
 * computed them (branches 3 and 4; zeros elsewhere). Returns 0, or -1 for a
 * bad index (outputs of later pairs are then unset). */
int ora_mlp_decide_many(const ora_tree *T, int64_t n, const int64_t *groups, const int64_t *cells,
                        const double *w, const double *mu, const double *sigma, const double *fmin,
                        const double *fmax, double tau, double theta_lo, double theta_hi, double theta_fb,
                        int bf16, int *open, int *branch, double *y, double *feat)
{
    mlp_rule R = {w, mu, sigma, fmin, fmax, tau, theta_lo, theta_hi, theta_fb, bf16};
    for (int64_t k = 0; k < n; ++k) {
        const int64_t g = groups[k], c = cells[k];
        if (g < 0 || g >= T->n_groups || c < 0 || c >= T->n_cells) return -1;
        open[k] = mlp_open(T, g, c, &R, &branch[k], &y[k]);
        if (feat) {
            if (branch[k] >= ORA_BR_FALLBACK) ora_mlp_features(T, g, c, feat + ORA_NF * k);
            else memset(feat + ORA_NF * k, 0, sizeof(double) * ORA_NF);
        }
    }
    return 0;
}

typedef struct {
    const ora_tree *T; double eps2, G; const mlp_rule *R;
    const int64_t *groups; int64_t ng; double *acc, *pot; int64_t *npp, *npc; int64_t next, n_mlp;
} mlpf_job;

static void *mlpf_worker(void *arg)
{
    mlpf_job *J = (mlpf_job *)arg;
    const ora_tree *T = J->T;
    vec cells = {0, 0, 0}, leaves = {0, 0, 0}, stack = {0, 0, 0};
    int64_t *tmp = NULL; int64_t tcap = 0;
    int64_t nm = 0;
    for (;;) {
        int64_t k = __atomic_fetch_add(&J->next, 1, __ATOMIC_RELAXED);
        if (k >= J->ng) break;
        const int64_t g = J->groups ? J->groups[k] : k, gc = T->group[g];
        cells.n = leaves.n = stack.n = 0;
        if (T->leaf[0]) vpush(&leaves, 0); else vpush(&stack, 0);
        while (stack.n) {
            int64_t node = stack.v[--stack.n];
            for (int o = 0; o < 8; ++o) {
                int64_t ch = T->child[8 * node + o];
                if (ch < 0) continue;
                int br; double y;
                if (mlp_open(T, g, ch, J->R, &br, &y)) {
                    if (T->leaf[ch]) vpush(&leaves, ch); else vpush(&stack, ch);
                } else vpush(&cells, ch);
                if (br == ORA_BR_NETWORK) ++nm;
            }
        }
        /* O6 summation order: cell list, then leaf list, each in key order */
        int64_t need = cells.n > leaves.n ? cells.n : leaves.n;
        if (need > tcap) { free(tmp); tcap = need; tmp = (int64_t *)malloc(sizeof(int64_t) * (size_t)tcap); }
        sort_by_key(cells.v, cells.n, T->key, tmp);
        sort_by_key(leaves.v, leaves.n, T->key, tmp);
        int64_t pp_src = 0;
        for (int64_t l = 0; l < leaves.n; ++l) pp_src += T->count[leaves.v[l]];
        for (int64_t a = T->first[gc]; a < T->first[gc] + T->count[gc]; ++a) {
            const int64_t i = T->idx[a];
            const double *xi = T->pos + 3 * i;
            double ax = 0, ay = 0, az = 0, phi = 0;
            for (int64_t e = 0; e < cells.n; ++e) {
                double ac[3], pc;
                ora_cell_field(T->com + 3 * cells.v[e], T->M[cells.v[e]], T->S + 6 * cells.v[e], xi, J->eps2, 1.0, ac, &pc);
                ax += ac[0]; ay += ac[1]; az += ac[2]; phi += pc;
            }
            for (int64_t e = 0; e < leaves.n; ++e) {
                const int64_t c = leaves.v[e];
                for (int64_t b = T->first[c]; b < T->first[c] + T->count[c]; ++b) {
                    const int64_t j = T->idx[b];
                    if (j == i) continue;
                    const double *xj = T->pos + 3 * j;
                    double dx = xj[0] - xi[0], dy = xj[1] - xi[1], dz = xj[2] - xi[2];
                    double r2 = dx * dx + dy * dy + dz * dz + J->eps2;
                    if (r2 == 0.0) continue;
                    double rinv = 1.0 / sqrt(r2);
                    double mr3 = T->mass[j] * rinv * rinv * rinv;
                    ax += mr3 * dx; ay += mr3 * dy; az += mr3 * dz;
                    phi -= T->mass[j] * rinv;
                }
            }
            J->acc[3 * i] = J->G * ax; J->acc[3 * i + 1] = J->G * ay; J->acc[3 * i + 2] = J->G * az;
            J->pot[i] = J->G * phi;
            if (J->npp) J->npp[i] = pp_src - 1;
            if (J->npc) J->npc[i] = cells.n;
        }
    }
    __atomic_fetch_add(&J->n_mlp, nm, __ATOMIC_RELAXED);
    free(cells.v); free(leaves.v); free(stack.v); free(tmp);
    return NULL;
}

/* Tree forces with the learned criterion (see mlp_open); arguments as
 * ora_forces plus the network, its thresholds and its precision (bf16 as for
 * ora_mlp_decide). Returns the number of network evaluations, or -1. */
int64_t ora_forces_mlp(const ora_tree *T, double eps, double G, const double *w, const double *mu,
                       const double *sigma, const double *fmin, const double *fmax, double tau, double theta_lo,
                       double theta_hi, double theta_fb, int bf16, const int64_t *groups, int64_t ng,
                       double *acc, double *pot, int64_t *npp, int64_t *npc, int nthreads)
{
    mlp_rule R = {w, mu, sigma, fmin, fmax, tau, theta_lo, theta_hi, theta_fb, bf16};
    mlpf_job J;
    memset(&J, 0, sizeof J);
    J.T = T; J.eps2 = eps * eps; J.G = G; J.R = &R;
    J.groups = groups; J.ng = groups ? ng : T->n_groups;
    J.acc = acc; J.pot = pot; J.npp = npp; J.npc = npc;
    run_threads(mlpf_worker, &J, nthreads);
    return J.n_mlp;
}

/* O6 on given lists: accelerations and potentials of group g's particles
 * (in the group's member order) from the cells of `cells` (multipole) and the
 * members of the leaves in `leaves` (direct, self excluded). Used to check a
 * walk whose lists come from elsewhere. */
void ora_forces_on_lists(const ora_tree *T, int64_t g, const int64_t *cells, int64_t nc, const int64_t *leaves,
                         int64_t nl, double eps, double G, double *acc, double *pot)
{
    const int64_t gc = T->group[g];
    const double eps2 = eps * eps;
    for (int64_t a = 0; a < T->count[gc]; ++a) {
        const int64_t i = T->idx[T->first[gc] + a];
        const double *xi = T->pos + 3 * i;
        double ax = 0, ay = 0, az = 0, phi = 0;
        for (int64_t e = 0; e < nc; ++e) {
            double ac[3], pc;
            ora_cell_field(T->com + 3 * cells[e], T->M[cells[e]], T->S + 6 * cells[e], xi, eps2, 1.0, ac, &pc);
            ax += ac[0]; ay += ac[1]; az += ac[2]; phi += pc;
        }
        for (int64_t e = 0; e < nl; ++e) {
            const int64_t c = leaves[e];
            for (int64_t b = T->first[c]; b < T->first[c] + T->count[c]; ++b) {
                const int64_t j = T->idx[b];
                if (j == i) continue;
                const double *xj = T->pos + 3 * j;
                double dx = xj[0] - xi[0], dy = xj[1] - xi[1], dz = xj[2] - xi[2];
                double r2 = dx * dx + dy * dy + dz * dz + eps2;
                if (r2 == 0.0) continue;
                double rinv = 1.0 / sqrt(r2);
                double mr3 = T->mass[j] * rinv * rinv * rinv;
                ax += mr3 * dx; ay += mr3 * dy; az += mr3 * dz;
                phi -= T->mass[j] * rinv;
            }
        }
        acc[3 * a] = G * ax; acc[3 * a + 1] = G * ay; acc[3 * a + 2] = G * az;
        pot[a] = G * phi;
    }
}
