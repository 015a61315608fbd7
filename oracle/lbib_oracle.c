/*
 * lbib_oracle.c -- plain FP64 CPU oracle of one LB-IB time step.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load this library.
 * It shares no source, header, table or constant generator with the CUDA
 * library: the D3Q19 set below is produced by enumeration, the fluid is
 * stored cell-major and streamed by "push" (the CUDA path pulls from a
 * direction-major array), and the mesh topology is found by brute force.
 *
 * Method: Cimrak, Gusenbauer, Jancigova, "An ESPResSo implementation of
 * elastic objects immersed in a fluid" (arXiv:1312.3426).  Every function
 * names the passage it follows.  Where the paper leaves a choice open the
 * readings are:
 *   - collision: single-relaxation-time BGK with relaxation time tau
 *     (Sec. 2 defers the operator to its references);
 *   - force term f_i: Guo's form, with the velocity u = (sum n e + G/2)/rho;
 *   - lattice node (i,j,k) sits at (i+1/2, j+1/2, k+1/2); with walls, the
 *     rows j=0 and j=ny-1 are solid and the halfway bounce-back planes are
 *     y=1 and y=ny-1; x and z are periodic (y too when walls are off);
 *   - drag (Eq. dragforce): the node receives xi (u - v) and the fluid the
 *     opposite, i.e. the paper's magnitude with the dissipative sign;
 *   - interpolation and spreading: trilinear weights (the weight of a
 *     corner is the volume of the cuboid between the point and the
 *     opposite corner); solid corners give u = 0 and receive no force;
 *   - Newton's law (Eq. newton): one update per LB step, v first, then X
 *     (symplectic Euler, dt = 1);
 *   - bending: per shared edge, each triangle pushes its own apex along its
 *     own inward unit normal with kb (theta - theta0)/theta0, and the two
 *     edge vertices take minus half of each;
 *   - global area: the centroid-to-vertex unit vector w of each triangle,
 *     summed over all triangles of the object;
 *   - volume: the object volume from the divergence theorem,
 *     V = -(1/6) sum A.(B x C) for inward-ordered triangles, taken relative
 *     to the object's first node.
 *
 * All arithmetic is FP64 and follows the printed formulas directly, loop by
 * loop, without blocking or fusion.  OpenMP (when available) splits only the
 * per-cell fluid loops, whose cells are independent, so results do not
 * depend on the thread count.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NQ 19

typedef struct {
    int nn, nt, ne;
    double *x;            /* rest coordinates after stretch, [nn][3] */
    int *tri;             /* [nt][3], inward-ordered as given */
    int *edge;            /* [ne][2], i < j, lexicographic */
    int *quad;            /* [ne][4] (a,b,c,d): edge (b,c) = edge[e];
                             (a,b,c) is a cyclic order of the triangle that
                             runs b->c, (d,c,b) of the one that runs c->b */
    double *L0, *theta0, *S0;
    double Sg0, V0;
    double ks, kb, kal, kag, kv;
    int nonlinear;
    int kal_altitude;     /* local area along the altitudes instead of centroid -> vertex */
} otpl;

typedef struct {
    int tid, first;
    double mass, fext[3];
} oobj;

/* Soft-sphere repulsion parameters: amplitude a, exponent n, cutoff rc. */
typedef struct {
    double a, n, rc;
} osoft;

typedef struct osim {
    int nx, ny, nz, walls;
    osoft rep_obj, rep_wall;  /* object-object and object-wall repulsion (a = 0: off) */
    int in_box[6];            /* velocity inlet cells x0..x1-1, y0..y1-1, z0..z1-1 (empty: off) */
    unsigned char *solid;     /* [ncell] obstacle cells (NULL: none) */
    double in_u[3];           /* prescribed velocity of the inlet */
    double tau, rho0, g[3], xi;
    long ncell;
    double *f, *fpost;        /* [ncell][NQ] */
    double *u, *rho;          /* [ncell][3], [ncell]: from the last collision */
    double *G;                /* [ncell][3]: force spread by the nodes */
    int E[NQ][3];
    double W[NQ];
    int OPP[NQ];
    int ntpl, nobj, nnode;
    otpl *tpl;
    oobj *obj;
    double *X, *V, *Fel;      /* [nnode][3] */
    double dropped[3];        /* momentum not spread because a corner was solid */
} osim;

/* ---------------------------------------------------------------- lattice */

/* D3Q19 lattice (Sec. 2): all e in {-1,0,1}^3 with
 * |e|^2 <= 2; weights 1/3, 1/18, 1/36 for |e|^2 = 0, 1, 2. */
static void lattice_init(osim *s)
{
    int q = 0;
    for (int ez = -1; ez <= 1; ++ez)
        for (int ey = -1; ey <= 1; ++ey)
            for (int ex = -1; ex <= 1; ++ex) {
                int n2 = ex * ex + ey * ey + ez * ez;
                if (n2 > 2) continue;
                s->E[q][0] = ex; s->E[q][1] = ey; s->E[q][2] = ez;
                s->W[q] = n2 == 0 ? 1.0 / 3.0 : (n2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
                ++q;
            }
    for (q = 0; q < NQ; ++q)
        for (int p = 0; p < NQ; ++p)
            if (s->E[p][0] == -s->E[q][0] && s->E[p][1] == -s->E[q][1] &&
                s->E[p][2] == -s->E[q][2])
                s->OPP[q] = p;
}

static long cell_index(const osim *s, int x, int y, int z)
{
    return ((long)z * s->ny + y) * s->nx + x;
}

static int is_solid_row(const osim *s, int y)
{
    return s->walls && (y <= 0 || y >= s->ny - 1);
}

/* Obstacle cells (the rhomboid obstacles of the Sec. 6 channel): solid like
 * the wall rows, i.e. never updated and reflecting what streams into them. */
static int is_solid_cell(const osim *s, long c, int y)
{
    return is_solid_row(s, y) || (s->solid && s->solid[c]);
}

static int wrap(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

/* ---------------------------------------------------------------- vectors */

static void sub3(const double *a, const double *b, double *r) { for (int k = 0; k < 3; ++k) r[k] = a[k] - b[k]; }
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double norm3(const double *a) { return sqrt(dot3(a, a)); }
static void cross3(const double *a, const double *b, double *r)
{
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}

/* ---------------------------------------------------------------- create */

osim *oracle_create(int nx, int ny, int nz, int walls, double tau, double rho0,
                    const double *g, double xi)
{
    if (nx < 1 || ny < 1 || nz < 1 || (walls && ny < 3) || tau <= 0.5) return NULL;
    osim *s = (osim *)calloc(1, sizeof(osim));
    s->nx = nx; s->ny = ny; s->nz = nz; s->walls = walls;
    s->tau = tau; s->rho0 = rho0; s->xi = xi;
    for (int k = 0; k < 3; ++k) s->g[k] = g ? g[k] : 0.0;
    s->ncell = (long)nx * ny * nz;
    s->f = (double *)calloc((size_t)s->ncell * NQ, sizeof(double));
    s->fpost = (double *)calloc((size_t)s->ncell * NQ, sizeof(double));
    s->u = (double *)calloc((size_t)s->ncell * 3, sizeof(double));
    s->rho = (double *)calloc((size_t)s->ncell, sizeof(double));
    s->G = (double *)calloc((size_t)s->ncell * 3, sizeof(double));
    lattice_init(s);
    return s;
}

void oracle_destroy(osim *s)
{
    if (!s) return;
    for (int t = 0; t < s->ntpl; ++t) {
        otpl *T = &s->tpl[t];
        free(T->x); free(T->tri); free(T->edge); free(T->quad);
        free(T->L0); free(T->theta0); free(T->S0);
    }
    free(s->tpl); free(s->obj); free(s->X); free(s->V); free(s->Fel);
    free(s->f); free(s->fpost); free(s->u); free(s->rho); free(s->G);
    free(s->solid);
    free(s);
}

int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_lattice(const osim *s, int *e, double *w)
{
    for (int q = 0; q < NQ; ++q) {
        for (int k = 0; k < 3; ++k) e[3 * q + k] = s->E[q][k];
        w[q] = s->W[q];
    }
}

/* ------------------------------------------------------- mesh geometry */

/* Triangle area S = |AB x AC| / 2 and unit normal along AB x AC, which is
 * the inward normal because mesh triangles are ordered so that AB x AC
 * points into the object (Sec. 5, template creation). */
static double tri_area_normal(const double *A, const double *B, const double *C, double *n)
{
    double ab[3], ac[3], c[3];
    sub3(B, A, ab); sub3(C, A, ac); cross3(ab, ac, c);
    double len = norm3(c);
    if (n) for (int k = 0; k < 3; ++k) n[k] = c[k] / len;
    return 0.5 * len;
}

/* Inner angle between triangles (a,b,c) and (d,c,b) at their common edge
 * (Sec. 4, bending force; closed objects use the angle measured through the
 * interior).  alpha is the
 * angle between the two inward normals; the edge is convex when d lies on
 * the inner side of the first triangle's plane, then theta = pi - alpha,
 * otherwise theta = pi + alpha (concave, theta > pi). */
static double dihedral(const double *a, const double *b, const double *c, const double *d,
                       double *n1, double *n2)
{
    tri_area_normal(a, b, c, n1);
    tri_area_normal(d, c, b, n2);
    double cr[3], db[3];
    cross3(n1, n2, cr);
    double alpha = atan2(norm3(cr), dot3(n1, n2));
    sub3(d, b, db);
    return dot3(db, n1) > 0.0 ? M_PI - alpha : M_PI + alpha;
}

/* Object surface S_g = sum of triangle areas (Sec. 4, global area) and
 * volume (Sec. 4, volume conservation).  The volume is the divergence
 * theorem sum; with inward-ordered triangles the outward normal is
 * -(AB x AC), hence the minus sign.  Coordinates are taken relative to the
 * first node of the object, a point that does not move with the sum. */
static void object_measures(const otpl *T, const double *X, double *Sg, double *V)
{
    const double *o = X;
    double sg = 0.0, v = 0.0;
    for (int t = 0; t < T->nt; ++t) {
        const double *A = X + 3 * T->tri[3 * t], *B = X + 3 * T->tri[3 * t + 1],
                     *C = X + 3 * T->tri[3 * t + 2];
        sg += tri_area_normal(A, B, C, NULL);
        double a[3], b[3], c[3], bc[3];
        sub3(A, o, a); sub3(B, o, b); sub3(C, o, c);
        cross3(b, c, bc);
        v += dot3(a, bc);
    }
    *Sg = sg;
    *V = -v / 6.0;
}

/* ------------------------------------------------------- templates */

/* Brute-force topology (Sec. 5 "Template creation"): every undirected edge
 * of the triangle list, i<j, sorted; for each edge, the triangle running
 * b->c gives the apex a and the triangle running c->b gives d.  Fails unless
 * every edge is used once in each direction (closed, consistently oriented
 * 2-manifold). */
static int build_topology(otpl *T)
{
    int maxe = 3 * T->nt;
    int *ed = (int *)malloc(sizeof(int) * 2 * maxe);
    int ne = 0;
    for (int t = 0; t < T->nt; ++t)
        for (int k = 0; k < 3; ++k) {
            int i = T->tri[3 * t + k], j = T->tri[3 * t + (k + 1) % 3];
            int lo = i < j ? i : j, hi = i < j ? j : i;
            int found = 0;
            for (int e = 0; e < ne; ++e)
                if (ed[2 * e] == lo && ed[2 * e + 1] == hi) { found = 1; break; }
            if (!found) { ed[2 * ne] = lo; ed[2 * ne + 1] = hi; ++ne; }
        }
    /* lexicographic insertion sort */
    for (int i = 1; i < ne; ++i) {
        int a = ed[2 * i], b = ed[2 * i + 1], j = i - 1;
        while (j >= 0 && (ed[2 * j] > a || (ed[2 * j] == a && ed[2 * j + 1] > b))) {
            ed[2 * (j + 1)] = ed[2 * j]; ed[2 * (j + 1) + 1] = ed[2 * j + 1]; --j;
        }
        ed[2 * (j + 1)] = a; ed[2 * (j + 1) + 1] = b;
    }
    int *qd = (int *)malloc(sizeof(int) * 4 * (ne ? ne : 1));
    for (int e = 0; e < ne; ++e) {
        int b = ed[2 * e], c = ed[2 * e + 1];
        int na = 0, nd = 0, a = -1, d = -1;
        for (int t = 0; t < T->nt; ++t)
            for (int k = 0; k < 3; ++k) {
                int i = T->tri[3 * t + k], j = T->tri[3 * t + (k + 1) % 3];
                int other = T->tri[3 * t + (k + 2) % 3];
                if (i == b && j == c) { a = other; ++na; }
                if (i == c && j == b) { d = other; ++nd; }
            }
        if (na != 1 || nd != 1) { free(ed); free(qd); return -3; }
        qd[4 * e] = a; qd[4 * e + 1] = b; qd[4 * e + 2] = c; qd[4 * e + 3] = d;
    }
    T->ne = ne; T->edge = ed; T->quad = qd;
    return 0;
}

/* oif_create_template (Sec. 5): geometry, stretch, moduli; relaxed lengths,
 * angles and areas are measured on the stretched template geometry. */
int oracle_template_create(osim *s, const double *xyz, int nn, const int *tri, int nt,
                           const double *stretch, double ks, double kb, double kal,
                           double kag, double kv, int nonlinear)
{
    if (nn < 4 || nt < 4) return -1;
    for (int i = 0; i < 3 * nt; ++i)
        if (tri[i] < 0 || tri[i] >= nn) return -3;
    s->tpl = (otpl *)realloc(s->tpl, sizeof(otpl) * (s->ntpl + 1));
    otpl *T = &s->tpl[s->ntpl];
    memset(T, 0, sizeof(*T));
    T->nn = nn; T->nt = nt;
    T->x = (double *)malloc(sizeof(double) * 3 * nn);
    for (int i = 0; i < nn; ++i)
        for (int k = 0; k < 3; ++k) T->x[3 * i + k] = xyz[3 * i + k] * (stretch ? stretch[k] : 1.0);
    T->tri = (int *)malloc(sizeof(int) * 3 * nt);
    memcpy(T->tri, tri, sizeof(int) * 3 * nt);
    int rc = build_topology(T);
    if (rc) { free(T->x); free(T->tri); return rc; }
    T->ks = ks; T->kb = kb; T->kal = kal; T->kag = kag; T->kv = kv; T->nonlinear = nonlinear;
    T->L0 = (double *)malloc(sizeof(double) * T->ne);
    T->theta0 = (double *)malloc(sizeof(double) * T->ne);
    T->S0 = (double *)malloc(sizeof(double) * nt);
    for (int e = 0; e < T->ne; ++e) {
        double d[3], n1[3], n2[3];
        sub3(T->x + 3 * T->edge[2 * e + 1], T->x + 3 * T->edge[2 * e], d);
        T->L0[e] = norm3(d);
        const int *q = T->quad + 4 * e;
        T->theta0[e] = dihedral(T->x + 3 * q[0], T->x + 3 * q[1], T->x + 3 * q[2],
                                T->x + 3 * q[3], n1, n2);
    }
    for (int t = 0; t < nt; ++t)
        T->S0[t] = tri_area_normal(T->x + 3 * tri[3 * t], T->x + 3 * tri[3 * t + 1],
                                   T->x + 3 * tri[3 * t + 2], NULL);
    object_measures(T, T->x, &T->Sg0, &T->V0);
    if (!(T->V0 > 0.0)) { /* triangles not ordered inward */
        free(T->x); free(T->tri); free(T->edge); free(T->quad);
        free(T->L0); free(T->theta0); free(T->S0);
        return -3;
    }
    return s->ntpl++;
}

int oracle_template_topology(const osim *s, int tid, int *edges, int *quads, double *L0,
                             double *theta0, double *S0, double *globals)
{
    if (tid < 0 || tid >= s->ntpl) return -2;
    const otpl *T = &s->tpl[tid];
    if (edges) memcpy(edges, T->edge, sizeof(int) * 2 * T->ne);
    if (quads) memcpy(quads, T->quad, sizeof(int) * 4 * T->ne);
    if (L0) memcpy(L0, T->L0, sizeof(double) * T->ne);
    if (theta0) memcpy(theta0, T->theta0, sizeof(double) * T->ne);
    if (S0) memcpy(S0, T->S0, sizeof(double) * T->nt);
    if (globals) { globals[0] = T->Sg0; globals[1] = T->V0; }
    return T->ne;
}

/* ------------------------------------------------------- objects */

/* oif_add_object (Sec. 5): copy the template, rotate by rx about x, then ry
 * about y, then rz about z (R = Rz Ry Rx), then translate by the origin. */
int oracle_object_add(osim *s, int tid, const double *origin, const double *rot, double mass)
{
    if (tid < 0 || tid >= s->ntpl || !(mass > 0.0)) return -1;
    const otpl *T = &s->tpl[tid];
    double cx = cos(rot[0]), sx = sin(rot[0]), cy = cos(rot[1]), sy = sin(rot[1]),
           cz = cos(rot[2]), sz = sin(rot[2]);
    double Rx[3][3] = {{1, 0, 0}, {0, cx, -sx}, {0, sx, cx}};
    double Ry[3][3] = {{cy, 0, sy}, {0, 1, 0}, {-sy, 0, cy}};
    double Rz[3][3] = {{cz, -sz, 0}, {sz, cz, 0}, {0, 0, 1}};
    double Ryx[3][3], R[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            Ryx[i][j] = 0.0;
            for (int k = 0; k < 3; ++k) Ryx[i][j] += Ry[i][k] * Rx[k][j];
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            R[i][j] = 0.0;
            for (int k = 0; k < 3; ++k) R[i][j] += Rz[i][k] * Ryx[k][j];
        }
    int first = s->nnode, n = s->nnode + T->nn;
    s->X = (double *)realloc(s->X, sizeof(double) * 3 * n);
    s->V = (double *)realloc(s->V, sizeof(double) * 3 * n);
    s->Fel = (double *)realloc(s->Fel, sizeof(double) * 3 * n);
    for (int i = 0; i < T->nn; ++i) {
        const double *p = T->x + 3 * i;
        for (int r = 0; r < 3; ++r) {
            s->X[3 * (first + i) + r] = R[r][0] * p[0] + R[r][1] * p[1] + R[r][2] * p[2] + origin[r];
            s->V[3 * (first + i) + r] = 0.0;
            s->Fel[3 * (first + i) + r] = 0.0;
        }
    }
    s->obj = (oobj *)realloc(s->obj, sizeof(oobj) * (s->nobj + 1));
    oobj *o = &s->obj[s->nobj];
    o->tid = tid; o->first = first; o->mass = mass;
    o->fext[0] = o->fext[1] = o->fext[2] = 0.0;
    s->nnode = n;
    return s->nobj++;
}

int oracle_object_nodes(const osim *s, int oid)
{
    if (oid < 0 || oid >= s->nobj) return -2;
    return s->tpl[s->obj[oid].tid].nn;
}

/* oif_object_set force (Sec. 5): the same ext_force on every node. */
int oracle_object_set_force(osim *s, int oid, const double *f)
{
    if (oid < 0 || oid >= s->nobj) return -2;
    for (int k = 0; k < 3; ++k) s->obj[oid].fext[k] = f[k];
    return 0;
}

/* oif_object_set mesh-nodes (Sec. 5): replace positions (velocities kept). */
int oracle_object_set_nodes(osim *s, int oid, const double *xyz)
{
    if (oid < 0 || oid >= s->nobj) return -2;
    const oobj *o = &s->obj[oid];
    memcpy(s->X + 3 * o->first, xyz, sizeof(double) * 3 * s->tpl[o->tid].nn);
    return 0;
}

int oracle_object_set_velocities(osim *s, int oid, const double *v)
{
    if (oid < 0 || oid >= s->nobj) return -2;
    const oobj *o = &s->obj[oid];
    memcpy(s->V + 3 * o->first, v, sizeof(double) * 3 * s->tpl[o->tid].nn);
    return 0;
}

int oracle_read_nodes(const osim *s, int oid, double *xyz, double *v)
{
    if (oid < 0 || oid >= s->nobj) return -2;
    const oobj *o = &s->obj[oid];
    int nn = s->tpl[o->tid].nn;
    if (xyz) memcpy(xyz, s->X + 3 * o->first, sizeof(double) * 3 * nn);
    if (v) memcpy(v, s->V + 3 * o->first, sizeof(double) * 3 * nn);
    return nn;
}

/* Current S_g and V of one object. */
int oracle_object_measures(const osim *s, int oid, double *out2)
{
    if (oid < 0 || oid >= s->nobj) return -2;
    const oobj *o = &s->obj[oid];
    object_measures(&s->tpl[o->tid], s->X + 3 * o->first, &out2[0], &out2[1]);
    return 0;
}

/* ------------------------------------------------------- elastic forces */

/* Sec. 4: the five OIF membrane forces of one object, accumulated into F
 * ([nn][3], not cleared here), from the node positions X of that object.
 * mask selects moduli: bit0 ks, bit1 kb, bit2 kal, bit3 kag, bit4 kv. */
static void membrane_forces(const otpl *T, const double *X, double *F, int mask)
{
    /* Stretching (Eq. stretching): F_s = ks kappa(lambda) dL/L0 n, with n the
     * unit vector between the endpoints, lambda = L/L0 and the neo-Hookean
     * kappa = (lambda^0.5 + lambda^-2.5)/(lambda + lambda^-3), or 1. */
    if (mask & 1)
        for (int e = 0; e < T->ne; ++e) {
            int a = T->edge[2 * e], b = T->edge[2 * e + 1];
            double d[3];
            sub3(X + 3 * b, X + 3 * a, d);
            double L = norm3(d), L0 = T->L0[e], lam = L / L0;
            double kap = T->nonlinear
                             ? (pow(lam, 0.5) + pow(lam, -2.5)) / (lam + pow(lam, -3.0))
                             : 1.0;
            double mag = T->ks * kap * (L - L0) / L0;
            for (int k = 0; k < 3; ++k) {
                F[3 * a + k] += mag * d[k] / L;
                F[3 * b + k] -= mag * d[k] / L;
            }
        }
    /* Bending: F_b = kb (theta - theta0)/theta0 n on the vertex off the
     * common edge, minus half of it on each of the two edge vertices. */
    if (mask & 2)
        for (int e = 0; e < T->ne; ++e) {
            const int *q = T->quad + 4 * e;
            double n1[3], n2[3];
            double th = dihedral(X + 3 * q[0], X + 3 * q[1], X + 3 * q[2], X + 3 * q[3], n1, n2);
            double sb = T->kb * (th - T->theta0[e]) / T->theta0[e];
            for (int k = 0; k < 3; ++k) {
                F[3 * q[0] + k] += sb * n1[k];
                F[3 * q[3] + k] += sb * n2[k];
                F[3 * q[1] + k] -= 0.5 * sb * (n1[k] + n2[k]);
                F[3 * q[2] + k] -= 0.5 * sb * (n1[k] + n2[k]);
            }
        }
    double Sg = 0.0, V = 0.0;
    if (mask & 24) object_measures(T, X, &Sg, &V);
    if (mask & 28)
        for (int t = 0; t < T->nt; ++t) {
            const int *v = T->tri + 3 * t;
            const double *A = X + 3 * v[0], *B = X + 3 * v[1], *C = X + 3 * v[2];
            double nin[3];
            double S = tri_area_normal(A, B, C, nin);
            double cen[3];
            for (int k = 0; k < 3; ++k) cen[k] = (A[k] + B[k] + C[k]) / 3.0;
            /* Local area: F_al = -kal (S - S0)/S w; global area:
             * F_ag = -kag (Sg - Sg0)/Sg w; w = unit(vertex - centroid). */
            double cl = (mask & 4) ? -T->kal * (S - T->S0[t]) / S : 0.0;
            double cg = (mask & 8) ? -T->kag * (Sg - T->Sg0) / Sg : 0.0;
            /* Volume: F_v = -kv (V - V0)/V0 S n_out, a third per vertex;
             * n_out = -n_in. */
            double cv = (mask & 16) ? T->kv * (V - T->V0) / T->V0 * S / 3.0 : 0.0;
            for (int j = 0; j < 3; ++j) {
                const double *P = X + 3 * v[j];
                double w[3];
                sub3(P, cen, w);
                double wl = norm3(w);
                double h[3], hl = 1.0;
                if (T->kal_altitude) {
                    /* the second direction of Sec. 4: along the altitude
                     * through the vertex, from the foot on the opposite
                     * edge to the vertex */
                    const double *Q = X + 3 * v[(j + 1) % 3], *R = X + 3 * v[(j + 2) % 3];
                    double e[3], d[3];
                    sub3(R, Q, e);
                    sub3(P, Q, d);
                    const double s = dot3(d, e) / dot3(e, e);
                    for (int k = 0; k < 3; ++k) h[k] = d[k] - s * e[k];
                    hl = norm3(h);
                } else {
                    for (int k = 0; k < 3; ++k) h[k] = w[k];
                    hl = wl;
                }
                for (int k = 0; k < 3; ++k)
                    F[3 * v[j] + k] += cl * h[k] / hl + cg * w[k] / wl + cv * nin[k];
            }
        }
}

/* Direction of the local-area force of template tid (Sec. 4 names two:
 * 0 = from the centroid to the vertex, 1 = along the vertex's altitude). */
int oracle_template_set_kal_direction(osim *s, int tid, int altitude)
{
    if (tid < 0 || tid >= s->ntpl) return -2;
    s->tpl[tid].kal_altitude = altitude ? 1 : 0;
    return 0;
}

/* Elastic forces of one object at its current nodes (cleared first). */
int oracle_membrane_forces(const osim *s, int oid, int mask, double *F)
{
    if (oid < 0 || oid >= s->nobj) return -2;
    const oobj *o = &s->obj[oid];
    const otpl *T = &s->tpl[o->tid];
    memset(F, 0, sizeof(double) * 3 * T->nn);
    membrane_forces(T, s->X + 3 * o->first, F, mask);
    return 0;
}

/* ------------------------------------------------------- coupling */

/* Sec. 2, IB method: the 8 lattice nodes around X and their trilinear
 * weights.  The weight of a corner is the volume of the cuboid spanned by
 * X and the diagonally opposite corner (unit cell), so the weights sum to
 * 1.  A point exactly on a lattice plane takes the lower node with weight 1.
 * Returns the cell index of each corner, or -1 for a solid corner. */
static void corners(const osim *s, const double *X, long *idx, double *w)
{
    int i0[3];
    double fr[3];
    for (int k = 0; k < 3; ++k) {
        double p = X[k] - 0.5;
        double fl = floor(p);
        i0[k] = (int)fl;
        fr[k] = p - fl;
    }
    for (int c = 0; c < 8; ++c) {
        int d[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
        double wc = 1.0;
        for (int k = 0; k < 3; ++k) wc *= d[k] ? fr[k] : 1.0 - fr[k];
        w[c] = wc;
        int ix = wrap(i0[0] + d[0], s->nx), iz = wrap(i0[2] + d[2], s->nz);
        int iy = i0[1] + d[1];
        if (s->walls) {
            if (iy < 0 || iy >= s->ny || is_solid_row(s, iy)) { idx[c] = -1; continue; }
        } else {
            iy = wrap(iy, s->ny);
        }
        idx[c] = cell_index(s, ix, iy, iz);
        if (s->solid && s->solid[idx[c]]) idx[c] = -1;
    }
}

/* Fluid velocity at X by linear interpolation (Sec. 2). */
static void interpolate_u(const osim *s, const double *X, double *u)
{
    long idx[8];
    double w[8];
    corners(s, X, idx, w);
    u[0] = u[1] = u[2] = 0.0;
    for (int c = 0; c < 8; ++c)
        if (idx[c] >= 0)
            for (int k = 0; k < 3; ++k) u[k] += w[c] * s->u[3 * idx[c] + k];
}

/* Eq. dragforce and Eq. newton for every node: F_d = xi (u(X) - v) acts on
 * the node, -F_d is spread to the fluid with the same weights, then
 * v += (F_el + F_d + F_ext)/m and X += v. */
static void couple_and_move(osim *s)
{
    for (int o = 0; o < s->nobj; ++o) {
        const oobj *ob = &s->obj[o];
        int nn = s->tpl[ob->tid].nn;
        for (int i = ob->first; i < ob->first + nn; ++i) {
            double *X = s->X + 3 * i, *V = s->V + 3 * i, *Fe = s->Fel + 3 * i;
            long idx[8];
            double w[8], u[3] = {0, 0, 0}, Fd[3];
            corners(s, X, idx, w);
            for (int c = 0; c < 8; ++c)
                if (idx[c] >= 0)
                    for (int k = 0; k < 3; ++k) u[k] += w[c] * s->u[3 * idx[c] + k];
            for (int k = 0; k < 3; ++k) Fd[k] = s->xi * (u[k] - V[k]);
            for (int c = 0; c < 8; ++c)
                for (int k = 0; k < 3; ++k) {
                    if (idx[c] >= 0) s->G[3 * idx[c] + k] -= w[c] * Fd[k];
                    else s->dropped[k] -= w[c] * Fd[k];
                }
            for (int k = 0; k < 3; ++k) {
                V[k] += (Fe[k] + Fd[k] + ob->fext[k]) / ob->mass;
                X[k] += V[k];
            }
        }
    }
}

/* ------------------------------------------------------- fluid */

/* Eq. lbequation, collision part, at every fluid cell: rho = sum n_i,
 * u = (sum n_i e_i + G/2)/rho (Guo), then BGK towards
 * f_eq = w rho (1 + 3 e.u + 4.5 (e.u)^2 - 1.5 u.u) plus the Guo force term
 * (1 - 1/(2 tau)) w [3 (e - u) + 9 (e.u) e].G, G = body force + IB force. */
static void collide(osim *s)
{
    const double tau = s->tau;
#pragma omp parallel for schedule(static)
    for (long c = 0; c < s->ncell; ++c) {
        int y = (int)((c / s->nx) % s->ny);
        if (is_solid_cell(s, c, y)) continue;
        const double *n = s->f + NQ * c;
        double *fp = s->fpost + NQ * c;
        double G[3], rho = 0.0, m[3] = {0.0, 0.0, 0.0}, u[3];
        for (int k = 0; k < 3; ++k) G[k] = s->g[k] + s->G[3 * c + k];
        for (int q = 0; q < NQ; ++q) {
            rho += n[q];
            for (int k = 0; k < 3; ++k) m[k] += n[q] * s->E[q][k];
        }
        for (int k = 0; k < 3; ++k) u[k] = (m[k] + 0.5 * G[k]) / rho;
        double uu = dot3(u, u);
        for (int q = 0; q < NQ; ++q) {
            double e[3] = {s->E[q][0], s->E[q][1], s->E[q][2]};
            double eu = dot3(e, u);
            double feq = s->W[q] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
            double Fq = 0.0;
            for (int k = 0; k < 3; ++k) Fq += (3.0 * (e[k] - u[k]) + 9.0 * eu * e[k]) * G[k];
            Fq *= s->W[q];
            fp[q] = n[q] - (n[q] - feq) / tau + (1.0 - 0.5 / tau) * Fq;
        }
        s->rho[c] = rho;
        for (int k = 0; k < 3; ++k) s->u[3 * c + k] = u[k];
    }
}

/* Eq. lbequation, propagation part (push): f_i(x + e_i) <- f*_i(x); a
 * population headed into a solid row is reflected into the opposite
 * direction of its own cell (halfway bounce-back of a resting wall, the
 * channel walls of Sec. 6). */
static void stream(osim *s)
{
#pragma omp parallel for schedule(static)
    for (long c = 0; c < s->ncell; ++c) {
        int x = (int)(c % s->nx), y = (int)((c / s->nx) % s->ny), z = (int)(c / ((long)s->nx * s->ny));
        if (is_solid_cell(s, c, y)) continue;
        for (int q = 0; q < NQ; ++q) {
            int tx = wrap(x + s->E[q][0], s->nx), tz = wrap(z + s->E[q][2], s->nz);
            int ty = y + s->E[q][1];
            if (s->walls && is_solid_row(s, ty)) {
                s->f[NQ * c + s->OPP[q]] = s->fpost[NQ * c + q];
                continue;
            }
            if (!s->walls) ty = wrap(ty, s->ny);
            const long t = cell_index(s, tx, ty, tz);
            if (s->solid && s->solid[t]) {  /* halfway bounce-back at an obstacle */
                s->f[NQ * c + s->OPP[q]] = s->fpost[NQ * c + q];
                continue;
            }
            s->f[NQ * t + q] = s->fpost[NQ * c + q];
        }
    }
}

/* lbfluid (Sec. 6): fluid at rest, f_i = w_i rho0, u = 0. */
void oracle_fluid_init(osim *s)
{
    for (long c = 0; c < s->ncell; ++c) {
        const int solid = s->solid && s->solid[c];
        for (int q = 0; q < NQ; ++q) s->f[NQ * c + q] = solid ? 0.0 : s->W[q] * s->rho0;
        s->rho[c] = solid ? 0.0 : s->rho0;
        s->u[3 * c] = s->u[3 * c + 1] = s->u[3 * c + 2] = 0.0;
    }
}

/* ------------------------------------------------------- repulsion */

/* Object-object and object-wall repulsion.  The example of Sec. 6 sets
 * "soft-sphere" interactions between the two objects and between each
 * object and the channel boundaries, with an amplitude a, an exponent n, a
 * cutoff and an offset; the paper does not print the potential.  Reading:
 * the usual soft-sphere pair potential V(r) = a r^-n for r < cutoff (offset
 * 0), so two nodes of different objects at distance r < cutoff push each
 * other apart along their separation with a force of magnitude a n
 * r^-(n+1); a node at distance d < cutoff from a wall plane (y = 1 or
 * y = ny-1) is pushed away from it with a n max(d, 1e-3)^-(n+1) (the floor
 * keeps a node that reached the plane finite).  Separations use the
 * minimum image in the periodic directions. */
static double soft_force(const osoft *p, double r) { return p->a * p->n * pow(r, -(p->n + 1.0)); }

static void repulsion(const osim *s, double *F)
{
    if (s->rep_obj.a != 0.0 && s->rep_obj.rc > 0.0) {
        const double L[3] = {s->nx, s->ny, s->nz};
        for (int oa = 0; oa < s->nobj; ++oa)
            for (int ob = oa + 1; ob < s->nobj; ++ob) {
                const oobj *A = &s->obj[oa], *B = &s->obj[ob];
                const int na = s->tpl[A->tid].nn, nb = s->tpl[B->tid].nn;
                for (int i = A->first; i < A->first + na; ++i)
                    for (int j = B->first; j < B->first + nb; ++j) {
                        double d[3];
                        sub3(s->X + 3 * i, s->X + 3 * j, d);
                        for (int k = 0; k < 3; ++k)
                            if (k != 1 || !s->walls) d[k] -= L[k] * round(d[k] / L[k]);
                        const double r = norm3(d);
                        if (!(r < s->rep_obj.rc) || r <= 0.0) continue;
                        const double f = soft_force(&s->rep_obj, r) / r;
                        for (int k = 0; k < 3; ++k) {
                            F[3 * i + k] += f * d[k];
                            F[3 * j + k] -= f * d[k];
                        }
                    }
            }
    }
    if (s->walls && s->rep_wall.a != 0.0 && s->rep_wall.rc > 0.0) {
        for (int i = 0; i < s->nnode; ++i) {
            const double y = s->X[3 * i + 1];
            const double dlo = y - 1.0, dhi = (s->ny - 1.0) - y;
            if (dlo < s->rep_wall.rc) F[3 * i + 1] += soft_force(&s->rep_wall, dlo > 1e-3 ? dlo : 1e-3);
            if (dhi < s->rep_wall.rc) F[3 * i + 1] -= soft_force(&s->rep_wall, dhi > 1e-3 ? dhi : 1e-3);
        }
    }
}

int oracle_set_repulsion(osim *s, const double *obj3, const double *wall3)
{
    if (!obj3 || !wall3) return -1;
    for (int k = 0; k < 3; ++k)
        if (!(obj3[k] >= 0.0) || !(wall3[k] >= 0.0)) return -1;
    s->rep_obj.a = obj3[0]; s->rep_obj.n = obj3[1]; s->rep_obj.rc = obj3[2];
    s->rep_wall.a = wall3[0]; s->rep_wall.n = wall3[1]; s->rep_wall.rc = wall3[2];
    return 0;
}

/* Repulsion forces of every node at the current positions (cleared first). */
void oracle_repulsion_forces(const osim *s, double *F)
{
    memset(F, 0, sizeof(double) * 3 * (size_t)s->nnode);
    repulsion(s, F);
}

/* ------------------------------------------------------- obstacles */

/* Marks obstacle cells from a [nz][ny][nx] byte mask (non-zero: solid);
 * NULL removes every obstacle.  Solid cells hold no fluid: their
 * populations and velocity are zero. */
int oracle_set_solid(osim *s, const unsigned char *mask)
{
    if (!mask) {
        free(s->solid);
        s->solid = NULL;
        return 0;
    }
    if (!s->solid) s->solid = (unsigned char *)calloc((size_t)s->ncell, 1);
    for (long c = 0; c < s->ncell; ++c) {
        s->solid[c] = mask[c] ? 1 : 0;
        if (s->solid[c]) {
            for (int q = 0; q < NQ; ++q) s->f[NQ * c + q] = s->fpost[NQ * c + q] = 0.0;
            s->u[3 * c] = s->u[3 * c + 1] = s->u[3 * c + 2] = 0.0;
            s->rho[c] = 0.0;
        }
    }
    return 0;
}

/* ------------------------------------------------------- inlet */

/* Velocity inlet (Sec. 6 example: before every integration step the fluid
 * velocity of the nodes of the inflow plane is set with "lbnode ... set u").
 * Reading: setting the velocity of a node replaces its populations by the
 * equilibrium at the node's own density and the prescribed velocity,
 * f_i = w_i rho (1 + 3 e.u + 4.5 (e.u)^2 - 1.5 u.u). */
int oracle_set_inlet(osim *s, const int *box, const double *u)
{
    for (int k = 0; k < 6; ++k) s->in_box[k] = box[k];
    for (int k = 0; k < 3; ++k) s->in_u[k] = u[k];
    return 0;
}

static void apply_inlet(osim *s)
{
    const int *b = s->in_box;
    const double uu = dot3(s->in_u, s->in_u);
    for (int z = b[4]; z < b[5]; ++z)
        for (int y = b[2]; y < b[3]; ++y)
            for (int x = b[0]; x < b[1]; ++x) {
                if (x < 0 || x >= s->nx || y < 0 || y >= s->ny || z < 0 || z >= s->nz) continue;
                if (is_solid_cell(s, cell_index(s, x, y, z), y)) continue;
                double *f = s->f + NQ * cell_index(s, x, y, z);
                double rho = 0.0;
                for (int q = 0; q < NQ; ++q) rho += f[q];
                for (int q = 0; q < NQ; ++q) {
                    const double e[3] = {s->E[q][0], s->E[q][1], s->E[q][2]};
                    const double eu = dot3(e, s->in_u);
                    f[q] = s->W[q] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
                }
            }
}

/* One full step, in the order: the velocity inlet (when set), object
 * measures and elastic forces (Sec. 4) plus the repulsion (Sec. 6
 * interactions, when set), interpolation, drag,
 * spreading and Newton update of the nodes (Sec. 2),
 * then collision and propagation of the fluid (Eq. lbequation) under the
 * body force plus the spread force. */
void oracle_step(osim *s, int nsteps)
{
    for (int it = 0; it < nsteps; ++it) {
        apply_inlet(s);
        memset(s->G, 0, sizeof(double) * 3 * s->ncell);
        if (s->nnode) memset(s->Fel, 0, sizeof(double) * 3 * s->nnode);
        for (int o = 0; o < s->nobj; ++o) {
            const oobj *ob = &s->obj[o];
            membrane_forces(&s->tpl[ob->tid], s->X + 3 * ob->first, s->Fel + 3 * ob->first, 31);
        }
        repulsion(s, s->Fel);
        couple_and_move(s);
        collide(s);
        stream(s);
    }
}

/* Membrane forces and node update against a frozen fluid velocity field
 * (no collision, no propagation); G keeps what the nodes spread. */
void oracle_step_nodes_only(osim *s, int nsteps)
{
    for (int it = 0; it < nsteps; ++it) {
        memset(s->G, 0, sizeof(double) * 3 * s->ncell);
        if (s->nnode) memset(s->Fel, 0, sizeof(double) * 3 * s->nnode);
        for (int o = 0; o < s->nobj; ++o) {
            const oobj *ob = &s->obj[o];
            membrane_forces(&s->tpl[ob->tid], s->X + 3 * ob->first, s->Fel + 3 * ob->first, 31);
        }
        repulsion(s, s->Fel);
        couple_and_move(s);
    }
}

/* ------------------------------------------------------- readouts */

/* Layouts: velocity [3][nz][ny][nx], density [nz][ny][nx], populations
 * [nz][ny][nx][19] in this file's direction order (oracle_lattice). */
void oracle_read_velocity(const osim *s, double *u)
{
    for (long c = 0; c < s->ncell; ++c)
        for (int k = 0; k < 3; ++k) u[k * s->ncell + c] = s->u[3 * c + k];
}

void oracle_set_velocity(osim *s, const double *u)
{
    for (long c = 0; c < s->ncell; ++c)
        for (int k = 0; k < 3; ++k) s->u[3 * c + k] = u[k * s->ncell + c];
}

void oracle_read_density(const osim *s, double *rho)
{
    memcpy(rho, s->rho, sizeof(double) * s->ncell);
}

void oracle_read_populations(const osim *s, double *f)
{
    memcpy(f, s->f, sizeof(double) * NQ * s->ncell);
}

void oracle_set_populations(osim *s, const double *f)
{
    memcpy(s->f, f, sizeof(double) * NQ * s->ncell);
}

void oracle_read_ib_force(const osim *s, double *G)
{
    for (long c = 0; c < s->ncell; ++c)
        for (int k = 0; k < 3; ++k) G[k * s->ncell + c] = s->G[3 * c + k];
}

void oracle_read_dropped(const osim *s, double *d)
{
    for (int k = 0; k < 3; ++k) d[k] = s->dropped[k];
}

/* Total fluid mass sum f and momentum sum f e over fluid cells. */
void oracle_fluid_totals(const osim *s, double *out4)
{
    double m = 0.0, p[3] = {0.0, 0.0, 0.0};
    for (long c = 0; c < s->ncell; ++c) {
        int y = (int)((c / s->nx) % s->ny);
        if (is_solid_cell(s, c, y)) continue;
        for (int q = 0; q < NQ; ++q) {
            m += s->f[NQ * c + q];
            for (int k = 0; k < 3; ++k) p[k] += s->f[NQ * c + q] * s->E[q][k];
        }
    }
    out4[0] = m; out4[1] = p[0]; out4[2] = p[1]; out4[3] = p[2];
}

/* Interpolated fluid velocity at an arbitrary point (test helper). */
void oracle_interpolate(const osim *s, const double *X, double *u)
{
    interpolate_u(s, X, u);
}

/* Current inner angle at every edge of one object (edge order of the
 * template topology). */
int oracle_object_edge_angles(const osim *s, int oid, double *theta)
{
    if (oid < 0 || oid >= s->nobj) return -2;
    const oobj *o = &s->obj[oid];
    const otpl *T = &s->tpl[o->tid];
    const double *X = s->X + 3 * o->first;
    for (int e = 0; e < T->ne; ++e) {
        const int *q = T->quad + 4 * e;
        double n1[3], n2[3];
        theta[e] = dihedral(X + 3 * q[0], X + 3 * q[1], X + 3 * q[2], X + 3 * q[3], n1, n2);
    }
    return T->ne;
}
