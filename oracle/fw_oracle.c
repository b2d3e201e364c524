/*
 * fw_oracle.c -- plain FP64 CPU oracle of the SDF contact substep (Factory, Sec. III).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the benchmark's
 * CPU-baseline leg, never by the product path.  Written for a reader checking it
 * against the paper: brute-force loops, FP64, steps in the paper's order.
 *
 * Readings of places where the paper is silent (each one a config field or a stated
 * constant, listed again in the project's design notes):
 *   R1 sign: phi < 0 inside the solid (Sec. III-A says only that the sign tells inside
 *      from outside).
 *   R2 grid: node-centred, dims^3 nodes spanning the padded bounding box (cubic).
 *   R3 gradient: the analytic gradient of the trilinear interpolant, i.e. the finite
 *      difference of neighbouring nodes weighted bilinearly in the other two axes
 *      ("gradients via finite-differencing", Sec. III-A).
 *   R4 a point outside the grid box, or with |grad| < 1e-12, makes no candidate.
 *   R5 candidate iff phi < contact_offset; the contact normal is the world-frame
 *      normalised SDF gradient of body B; the point on B is x_A - phi n.
 *   R6 Algorithm 1: batches of batch_size samples in sample order; Assign joins the
 *      existing patch of largest n.n_P if that is >= cos_patch (ties: lowest patch);
 *      FindDeepest = min phi (ties: lowest sample); BinReduce joins remaining
 *      candidates with n.n_best >= cos_patch; normals only, as Algorithm 1 states.
 *   R7 patch contents: slot 0 the deepest member, slots 1..6 the members extreme
 *      along u_k = cos(k pi/3) t1 + sin(k pi/3) t2 (k = 0..5) from the anchor; emitted
 *      contacts are the distinct slot members in slot order, patches in list order.
 *   R8 AddPatch: append below max_patches; at capacity replace the patch with the most
 *      similar normal iff M(new) > M(old), M = -phi_deepest + sqrt(area of the
 *      direction-slot polygon in the patch plane).
 *   R9 solver: velocity-level projected Gauss-Seidel; per contact the normal row
 *      (lambda_n >= 0) then the two friction rows projected jointly on the disk
 *      |lambda_t| <= mu lambda_n; bias phi/hs when phi > 0 (speculative), baumgarte *
 *      phi/hs otherwise; no warm start; mu of a pair = sqrt(mu_a mu_b).
 *   R10 integration: semi-implicit Euler on the centre of mass and
 *      q <- normalize(q + hs/2 (omega,0) q); |omega| clamped to max_angvel if set.
 *   R11 tangent basis: t1 = normalize(n x e_x) if |n_x| < 0.57735 else
 *      normalize(n x e_y); t2 = n x t1.
 *   R15 per-triangle generator (contact_gen = 1; Sec. III-A: one contact per face of the
 *      point body's mesh by local minimisation with projected gradient descent and
 *      adaptive steps): in body B's frame, start at the face centroid with step length
 *      s = half the longest edge; each of tri_iters steps moves against the gradient's
 *      in-plane part by s, projects onto the face (closest point), and is accepted when
 *      phi decreases (then s *= 1.5), else rejected (s *= 0.5); the descent stops when
 *      the in-plane gradient is below 1e-9.  A face whose centroid is outside the grid,
 *      or whose final gradient vanishes, makes no candidate; trial points outside the
 *      grid are rejected.  The candidate index is the triangle index, Generate batches
 *      are batch_size triangles.
 *   R17 narrow-band bricked storage (sdf_band > 0; the Limitations section plans sparse
 *      SDF storage against the grids' memory footprint without fixing a scheme): cells are grouped
 *      in bricks of 8^3; a brick is stored iff one node of its cells has |phi| <= band
 *      (band = sdf_band voxels, in float32: sdf_band * h) or its nodes change sign, the
 *      decision taken on the float32 node values.  A query in a cell of a brick that is
 *      not stored returns phi = +band (all its nodes positive) or -band (all negative)
 *      with a zero gradient, so it makes no candidate (R4).  Since a trilinear value is a
 *      convex combination of its cell's corners, every point with |phi| <= band lies in
 *      a stored brick and reads the dense value there.
 *   R18 Jacobi solver (solver = 1; the paper's solver comparison sizes a Jacobi solver at
 *      8 substeps x 64 iterations without stating its update): a sweep computes every
 *      contact's block update -- the normal row, then the friction rows with that
 *      contact's own normal change applied, projected on the disk -- from the velocities
 *      at the sweep's start, then takes all of them with the weight omega = 1 / (number
 *      of contacts that can act), impulses and velocities alike (a convex step towards
 *      each block's answer, so impulses stay in the friction cone).
 */
#include "fw_oracle.h"

#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------------------ */
/* small vector helpers                                                                   */
/* ------------------------------------------------------------------------------------ */
static void v_sub(const double a[3], const double b[3], double r[3]) { r[0] = a[0] - b[0]; r[1] = a[1] - b[1]; r[2] = a[2] - b[2]; }
static void v_add(const double a[3], const double b[3], double r[3]) { r[0] = a[0] + b[0]; r[1] = a[1] + b[1]; r[2] = a[2] + b[2]; }
static void v_scale(const double a[3], double s, double r[3]) { r[0] = a[0] * s; r[1] = a[1] * s; r[2] = a[2] * s; }
static void v_axpy(double s, const double a[3], double r[3]) { r[0] += s * a[0]; r[1] += s * a[1]; r[2] += s * a[2]; }
static double v_dot(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void v_cross(const double a[3], const double b[3], double r[3]) {
    double x = a[1] * b[2] - a[2] * b[1], y = a[2] * b[0] - a[0] * b[2], z = a[0] * b[1] - a[1] * b[0];
    r[0] = x; r[1] = y; r[2] = z;
}
static double v_norm(const double a[3]) { return sqrt(v_dot(a, a)); }
static void m_vec(const double M[9], const double v[3], double r[3]) {
    double x = M[0] * v[0] + M[1] * v[1] + M[2] * v[2];
    double y = M[3] * v[0] + M[4] * v[1] + M[5] * v[2];
    double z = M[6] * v[0] + M[7] * v[1] + M[8] * v[2];
    r[0] = x; r[1] = y; r[2] = z;
}
static void m_mul(const double A[9], const double B[9], double C[9]) {
    double T[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            T[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
    memcpy(C, T, sizeof T);
}
static void m_transpose(const double A[9], double B[9]) {
    double T[9] = {A[0], A[3], A[6], A[1], A[4], A[7], A[2], A[5], A[8]};
    memcpy(B, T, sizeof T);
}
static int m_inverse(const double A[9], double B[9]) {
    double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
    double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    if (det == 0.0) return -1;
    double id = 1.0 / det;
    B[0] = c00 * id; B[1] = (A[2] * A[7] - A[1] * A[8]) * id; B[2] = (A[1] * A[5] - A[2] * A[4]) * id;
    B[3] = c01 * id; B[4] = (A[0] * A[8] - A[2] * A[6]) * id; B[5] = (A[2] * A[3] - A[0] * A[5]) * id;
    B[6] = c02 * id; B[7] = (A[1] * A[6] - A[0] * A[7]) * id; B[8] = (A[0] * A[4] - A[1] * A[3]) * id;
    return 0;
}
/* rotation matrix of a unit quaternion (x, y, z, w) */
static void q_to_m(const double q[4], double R[9]) {
    double x = q[0], y = q[1], z = q[2], w = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - z * w);     R[2] = 2 * (x * z + y * w);
    R[3] = 2 * (x * y + z * w);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - x * w);
    R[6] = 2 * (x * z - y * w);     R[7] = 2 * (y * z + x * w);     R[8] = 1 - 2 * (x * x + y * y);
}
static void q_normalize(double q[4]) {
    double s = 1.0 / sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int i = 0; i < 4; ++i) q[i] *= s;
}
static void load3(const float *f, double d[3]) { d[0] = f[0]; d[1] = f[1]; d[2] = f[2]; }

/* ------------------------------------------------------------------------------------ */
/* closest point on a triangle (Ericson 5.1.5: classify p against the Voronoi regions   */
/* of the vertices, then of the edges, else project onto the face)                        */
/* ------------------------------------------------------------------------------------ */
int or_closest_point_triangle(const double p[3], const double a[3], const double b[3],
                              const double c[3], double q[3]) {
    double ab[3], ac[3], ap[3], bp[3], cp[3];
    v_sub(b, a, ab); v_sub(c, a, ac); v_sub(p, a, ap);
    double d1 = v_dot(ab, ap), d2 = v_dot(ac, ap);
    if (d1 <= 0.0 && d2 <= 0.0) { memcpy(q, a, 3 * sizeof(double)); return 1; }
    v_sub(p, b, bp);
    double d3 = v_dot(ab, bp), d4 = v_dot(ac, bp);
    if (d3 >= 0.0 && d4 <= d3) { memcpy(q, b, 3 * sizeof(double)); return 2; }
    v_sub(p, c, cp);
    double d5 = v_dot(ab, cp), d6 = v_dot(ac, cp);
    if (d6 >= 0.0 && d5 <= d6) { memcpy(q, c, 3 * sizeof(double)); return 3; }
    /* edge regions: the barycentric coordinate of the opposite vertex is <= 0 */
    double vc = d1 * d4 - d3 * d2;          /* weight of c */
    if (vc <= 0.0 && d1 >= 0.0 && d3 <= 0.0) {
        double t = d1 / (d1 - d3);
        q[0] = a[0] + t * ab[0]; q[1] = a[1] + t * ab[1]; q[2] = a[2] + t * ab[2];
        return 4;
    }
    double va = d3 * d6 - d5 * d4;          /* weight of a */
    if (va <= 0.0 && (d4 - d3) >= 0.0 && (d5 - d6) >= 0.0) {
        double t = (d4 - d3) / ((d4 - d3) + (d5 - d6));
        q[0] = b[0] + t * (c[0] - b[0]); q[1] = b[1] + t * (c[1] - b[1]); q[2] = b[2] + t * (c[2] - b[2]);
        return 5;
    }
    double vb = d5 * d2 - d1 * d6;          /* weight of b */
    if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) {
        double t = d2 / (d2 - d6);
        q[0] = a[0] + t * ac[0]; q[1] = a[1] + t * ac[1]; q[2] = a[2] + t * ac[2];
        return 6;
    }
    double s = 1.0 / (va + vb + vc);
    double v = vb * s, w = vc * s;
    q[0] = a[0] + v * ab[0] + w * ac[0];
    q[1] = a[1] + v * ab[1] + w * ac[1];
    q[2] = a[2] + v * ab[2] + w * ac[2];
    return 0;
}

/* Van Oosterom & Strackee (1983): tan(Omega/2) = det[a b c] /
 * (|a||b||c| + (a.b)|c| + (b.c)|a| + (c.a)|b|), vectors taken from p. */
double or_solid_angle(const double p[3], const double a[3], const double b[3], const double c[3]) {
    double A[3], B[3], C[3], bxc[3];
    v_sub(a, p, A); v_sub(b, p, B); v_sub(c, p, C);
    double la = v_norm(A), lb = v_norm(B), lc = v_norm(C);
    v_cross(B, C, bxc);
    double num = v_dot(A, bxc);
    double den = la * lb * lc + v_dot(A, B) * lc + v_dot(B, C) * la + v_dot(C, A) * lb;
    return 2.0 * atan2(num, den);
}

double or_winding_number(const double p[3], const float *V, const int *T, int nt) {
    double sum = 0.0;
    for (int t = 0; t < nt; ++t) {
        double a[3], b[3], c[3];
        load3(V + 3 * T[3 * t], a); load3(V + 3 * T[3 * t + 1], b); load3(V + 3 * T[3 * t + 2], c);
        sum += or_solid_angle(p, a, b, c);
    }
    return sum / (4.0 * M_PI);
}

double or_point_mesh_distance(const double p[3], const float *V, const int *T, int nt) {
    double best = INFINITY;
    for (int t = 0; t < nt; ++t) {
        double a[3], b[3], c[3], q[3], d[3];
        load3(V + 3 * T[3 * t], a); load3(V + 3 * T[3 * t + 1], b); load3(V + 3 * T[3 * t + 2], c);
        or_closest_point_triangle(p, a, b, c, q);
        v_sub(p, q, d);
        double dd = v_dot(d, d);
        if (dd < best) best = dd;
    }
    return sqrt(best);
}

/* ------------------------------------------------------------------------------------ */
/* mass properties: sum over tetrahedra (0, a, b, c) of signed volume, first and second */
/* moments.  For a tetrahedron with vertices p0..p3 the second moment is                  */
/*   int x x^T dV = V/20 (sum_i p_i p_i^T + (sum_i p_i)(sum_i p_i)^T).                     */
/* ------------------------------------------------------------------------------------ */
void or_mass_properties(const float *V, const int *T, int nt, double density,
                        double *mass, double com[3], double inertia[9]) {
    double vol = 0.0, m1[3] = {0, 0, 0}, C[9] = {0};
    for (int t = 0; t < nt; ++t) {
        double a[3], b[3], c[3], bxc[3];
        load3(V + 3 * T[3 * t], a); load3(V + 3 * T[3 * t + 1], b); load3(V + 3 * T[3 * t + 2], c);
        v_cross(b, c, bxc);
        double v = v_dot(a, bxc) / 6.0;
        double s[3] = {a[0] + b[0] + c[0], a[1] + b[1] + c[1], a[2] + b[2] + c[2]};
        vol += v;
        for (int i = 0; i < 3; ++i) m1[i] += v * s[i] / 4.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                C[3 * i + j] += v / 20.0 * (a[i] * a[j] + b[i] * b[j] + c[i] * c[j] + s[i] * s[j]);
    }
    double m = density * vol;
    double cm[3] = {m1[0] / vol, m1[1] / vol, m1[2] / vol};
    /* inertia about the origin: rho (tr(C) I - C); shift to the centre of mass */
    double tr = C[0] + C[4] + C[8];
    double c2 = v_dot(cm, cm);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double Io = density * ((i == j ? tr : 0.0) - C[3 * i + j]);
            double sh = m * ((i == j ? c2 : 0.0) - cm[i] * cm[j]);
            inertia[3 * i + j] = Io - sh;
        }
    *mass = m;
    memcpy(com, cm, sizeof cm);
}

/* ------------------------------------------------------------------------------------ */
/* grid placement (R2): padded bounding box, h = L/(res-1) with L the longest padded    */
/* extent; every value is rounded to float32 because the grid is stored in float32;     */
/* cubic: res^3 nodes centred on the box centre.                                          */
/* ------------------------------------------------------------------------------------ */
void or_grid_params(const float *V, int nv, int res, float pad, int cubic,
                    float lo[3], float *h, int dims[3]) {
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = 0; i < nv; ++i)
        for (int a = 0; a < 3; ++a) {
            double x = V[3 * i + a];
            if (x < mn[a]) mn[a] = x;
            if (x > mx[a]) mx[a] = x;
        }
    double ext[3], L = 0.0;
    for (int a = 0; a < 3; ++a) {
        ext[a] = mx[a] - mn[a] + 2.0 * (double)pad;
        if (ext[a] > L) L = ext[a];
    }
    float hf = (float)(L / (double)(res - 1));
    *h = hf;
    for (int a = 0; a < 3; ++a) {
        int n = res;
        if (!cubic) n = (int)ceil(ext[a] / (double)hf - 1e-9) + 1;
        dims[a] = n;
        lo[a] = (float)(0.5 * (mn[a] + mx[a]) - (double)hf * (double)(n - 1) * 0.5);
    }
}

static double node_phi(const double x[3], const float *V, const int *T, int nt) {
    double d = or_point_mesh_distance(x, V, T, nt);
    if (d == 0.0) return 0.0;
    double w = or_winding_number(x, V, T, nt);
    return (w > 0.5) ? -d : d;        /* R1 */
}

/* threads of one parallel region: n_threads, or the OpenMP default when n_threads <= 0
 * (set per region, never process-wide, so one world's setting cannot slow another's) */
static int team_size(int n_threads) {
#ifdef _OPENMP
    return n_threads > 0 ? n_threads : omp_get_max_threads();
#else
    (void)n_threads;
    return 1;
#endif
}

void or_bake_nodes(const float *V, const int *T, int nt, const float lo[3], float h,
                   const int dims[3], const long long *nodes, long long n_nodes,
                   double *phi, int n_threads) {
    long long total = nodes ? n_nodes : (long long)dims[0] * dims[1] * dims[2];
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) num_threads(team_size(n_threads))
#endif
    for (long long q = 0; q < total; ++q) {
        long long id = nodes ? nodes[q] : q;
        long long i = id % dims[0], j = (id / dims[0]) % dims[1], k = id / ((long long)dims[0] * dims[1]);
        double x[3] = {(double)lo[0] + (double)i * (double)h, (double)lo[1] + (double)j * (double)h,
                       (double)lo[2] + (double)k * (double)h};
        phi[q] = node_phi(x, V, T, nt);
    }
}

/* ------------------------------------------------------------------------------------ */
/* trilinear value and gradient (Sec. III-A; R3, R4)                                     */
/* ------------------------------------------------------------------------------------ */
#define BRICK 8                       /* cells per brick edge (R17) */
#define BRICK_UNKNOWN (-3)

typedef struct {
    double lo[3], h;
    int dims[3];
    double *val;          /* nx*ny*nz */
    unsigned char *done;  /* lazy bake: 1 when val is set */
    int lazy;
    float band;           /* R17: narrow band (m, float32); 0 = dense storage */
    int bdims[3];         /* bricks per axis */
    signed char *bstate;  /* per brick: 1 stored, -1 out of band outside, -2 inside, unknown */
} grid_t;

static long long gidx(const grid_t *g, int i, int j, int k) {
    return ((long long)k * g->dims[1] + j) * g->dims[0] + i;
}

static long long brick_index(const grid_t *g, int ci, int cj, int ck) {
    return ((long long)(ck / BRICK) * g->bdims[1] + cj / BRICK) * g->bdims[0] + ci / BRICK;
}

/* R17: the state of brick (bi, bj, bk) from its nodes (those of its cells), or unknown
 * while a lazy grid has not baked all of them */
static signed char brick_state(const grid_t *g, int bi, int bj, int bk) {
    const int b[3] = {bi, bj, bk};
    int n0[3], n1[3];
    for (int a = 0; a < 3; ++a) {
        n0[a] = b[a] * BRICK;
        n1[a] = n0[a] + BRICK;                                   /* last node of its last cell */
        if (n1[a] > g->dims[a] - 1) n1[a] = g->dims[a] - 1;
    }
    int near = 0, pos = 0, neg = 0;
    for (int k = n0[2]; k <= n1[2]; ++k)
        for (int j = n0[1]; j <= n1[1]; ++j)
            for (int i = n0[0]; i <= n1[0]; ++i) {
                const long long id = gidx(g, i, j, k);
                if (g->lazy && g->done[id] != 1) return BRICK_UNKNOWN;
                const float v = (float)g->val[id];
                if (fabsf(v) <= g->band) near = 1;
                if (v < 0.0f) neg = 1; else pos = 1;
            }
    if (near || (pos && neg)) return 1;
    return neg ? -2 : -1;
}

/* R17: set up the brick table of a grid (band in voxels); states of bricks whose nodes are
 * all known are computed now, the rest when a lazy bake completes them */
static void grid_set_band(grid_t *g, float band_voxels) {
    free(g->bstate);
    g->bstate = NULL;
    g->band = 0.0f;
    if (!(band_voxels > 0.0f)) return;
    g->band = band_voxels * (float)g->h;
    long long nb = 1;
    for (int a = 0; a < 3; ++a) {
        g->bdims[a] = (g->dims[a] - 1 + BRICK - 1) / BRICK;
        nb *= g->bdims[a];
    }
    g->bstate = (signed char *)malloc((size_t)nb);
    for (long long b = 0; b < nb; ++b) g->bstate[b] = BRICK_UNKNOWN;
    for (int bk = 0; bk < g->bdims[2]; ++bk)
        for (int bj = 0; bj < g->bdims[1]; ++bj)
            for (int bi = 0; bi < g->bdims[0]; ++bi)
                g->bstate[brick_index(g, bi * BRICK, bj * BRICK, bk * BRICK)] = brick_state(g, bi, bj, bk);
}

/* returns 0 when the point is outside the grid box; *margin = distance (m) to the box */
static int trilinear(const grid_t *g, const double x[3], double *phi, double grad[3], double *margin) {
    double u[3], f[3];
    int c[3];
    double mg = INFINITY;
    for (int a = 0; a < 3; ++a) {
        u[a] = (x[a] - g->lo[a]) / g->h;
        double m = fmin(u[a], (double)(g->dims[a] - 1) - u[a]) * g->h;
        if (fabs(m) < mg) mg = fabs(m);
    }
    if (margin) *margin = mg;
    for (int a = 0; a < 3; ++a)
        if (!(u[a] >= 0.0 && u[a] <= (double)(g->dims[a] - 1))) return 0;
    for (int a = 0; a < 3; ++a) {
        int ci = (int)floor(u[a]);
        if (ci > g->dims[a] - 2) ci = g->dims[a] - 2;
        if (ci < 0) ci = 0;
        c[a] = ci;
        f[a] = u[a] - ci;
    }
    if (g->band > 0.0f) {   /* R17: a brick out of the band answers +-band, no gradient */
        const signed char st = g->bstate[brick_index(g, c[0], c[1], c[2])];
        if (st == -1 || st == -2) {
            *phi = st == -1 ? (double)g->band : -(double)g->band;
            grad[0] = grad[1] = grad[2] = 0.0;
            return 1;
        }
    }
    double v[2][2][2];
    for (int dk = 0; dk < 2; ++dk)
        for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di)
                v[dk][dj][di] = g->val[gidx(g, c[0] + di, c[1] + dj, c[2] + dk)];
    double wx[2] = {1 - f[0], f[0]}, wy[2] = {1 - f[1], f[1]}, wz[2] = {1 - f[2], f[2]};
    double p = 0, gx = 0, gy = 0, gz = 0;
    for (int dk = 0; dk < 2; ++dk)
        for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di)
                p += wx[di] * wy[dj] * wz[dk] * v[dk][dj][di];
    for (int dk = 0; dk < 2; ++dk)
        for (int dj = 0; dj < 2; ++dj) gx += wy[dj] * wz[dk] * (v[dk][dj][1] - v[dk][dj][0]);
    for (int dk = 0; dk < 2; ++dk)
        for (int di = 0; di < 2; ++di) gy += wx[di] * wz[dk] * (v[dk][1][di] - v[dk][0][di]);
    for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di) gz += wx[di] * wy[dj] * (v[1][dj][di] - v[0][dj][di]);
    *phi = p;
    grad[0] = gx / g->h; grad[1] = gy / g->h; grad[2] = gz / g->h;
    return 1;
}

void or_query(const double *grid, const float lo[3], float h, const int dims[3],
              const float *pts, int n, double *phi, double *grad, int *valid) {
    grid_t g;
    memset(&g, 0, sizeof g);
    for (int a = 0; a < 3; ++a) { g.lo[a] = lo[a]; g.dims[a] = dims[a]; }
    g.h = h;
    g.val = (double *)grid;
    for (int i = 0; i < n; ++i) {
        double x[3], gr[3], p;
        load3(pts + 3 * i, x);
        int ok = trilinear(&g, x, &p, gr, NULL);
        valid[i] = ok;
        phi[i] = ok ? p : 0.0;
        for (int a = 0; a < 3; ++a) grad[3 * i + a] = ok ? gr[a] : 0.0;
    }
}

/* or_query on a grid held in bricked storage (R17); *n_stored, *n_bricks: the bricks kept */
void or_query_band(const double *grid, const float lo[3], float h, const int dims[3], float band_voxels,
                   const float *pts, int n, double *phi, double *grad, int *valid, int *n_stored, int *n_bricks) {
    grid_t g;
    memset(&g, 0, sizeof g);
    for (int a = 0; a < 3; ++a) { g.lo[a] = lo[a]; g.dims[a] = dims[a]; }
    g.h = h;
    g.val = (double *)grid;
    grid_set_band(&g, band_voxels);
    for (int i = 0; i < n; ++i) {
        double x[3], gr[3], p;
        load3(pts + 3 * i, x);
        int ok = trilinear(&g, x, &p, gr, NULL);
        valid[i] = ok;
        phi[i] = ok ? p : 0.0;
        for (int a = 0; a < 3; ++a) grad[3 * i + a] = ok ? gr[a] : 0.0;
    }
    int ns = 0, nb = 0;
    if (g.bstate) {
        nb = g.bdims[0] * g.bdims[1] * g.bdims[2];
        for (int b = 0; b < nb; ++b) ns += g.bstate[b] == 1;
    }
    if (n_stored) *n_stored = ns;
    if (n_bricks) *n_bricks = nb;
    free(g.bstate);
}

/* ------------------------------------------------------------------------------------ */
/* world                                                                                  */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    float *V; int nv; int *T; int nt;
    float *S; int ns;
    double density, mass, com[3], I[9];
    double radius;              /* bounding sphere about the asset origin (vertices, samples) */
    int has_grid;
    grid_t grid;
} asset_t;

typedef struct {
    int asset, type;
    double mass, mu;
    double invm, Ib[9], Ib_inv[9], com_b[3];
    double axis[3], force[3], torque[3];
    double p[3], q[4], v[3], w[3];
} body_t;

typedef struct { int a, b; double mu; int color; } pair_t;   /* global body ids; colour (piles) */

typedef struct {
    or_contact *c; int n, cap;
    double m_len, m_dot;        /* margins of the last detection of this pair */
    int n_patches;
} pair_contacts_t;

typedef struct {
    int first_body, n_bodies, first_pair, n_pairs;
    /* piles (R20): the pairs come from a broad phase at every detection */
    int pile;
    pair_t *dp; pair_contacts_t *dpc; int ndp, cap_dp;
} env_t;

struct or_world {
    or_config cfg;
    asset_t *assets; int n_assets, cap_assets;
    body_t *bodies; int n_bodies;
    pair_t *pairs; int n_pairs;
    env_t *envs; int n_envs;
    pair_contacts_t *pc;
    double *env_mlen, *env_mdot;
    double **imp; int *imp_n;               /* per env friction record */
    double bake_seconds;                    /* wall time spent in lazy SDF bakes */
    struct diff_tape *tape;                 /* decisions of the last recorded rollout */
};

static void diff_tape_free(or_world *w);

or_world *or_create(const or_config *cfg) {
    or_world *w = (or_world *)calloc(1, sizeof(or_world));
    w->cfg = *cfg;
    return w;
}

void or_set_threads(or_world *w, int n_threads) {
    if (w) w->cfg.n_threads = n_threads;
}

void or_destroy(or_world *w) {
    if (!w) return;
    for (int i = 0; i < w->n_assets; ++i) {
        asset_t *a = &w->assets[i];
        free(a->V); free(a->T); free(a->S); free(a->grid.val); free(a->grid.done); free(a->grid.bstate);
    }
    for (int i = 0; i < w->n_pairs; ++i) free(w->pc[i].c);
    for (int e = 0; e < w->n_envs; ++e) {
        for (int i = 0; i < w->envs[e].cap_dp; ++i) free(w->envs[e].dpc[i].c);
        free(w->envs[e].dp); free(w->envs[e].dpc);
    }
    free(w->assets); free(w->bodies); free(w->pairs); free(w->envs); free(w->pc);
    diff_tape_free(w);
    for (int e = 0; e < w->n_envs; ++e) free(w->imp[e]);
    free(w->env_mlen); free(w->env_mdot); free(w->imp); free(w->imp_n);
    free(w);
}

int or_add_asset(or_world *w, const float *V, int nv, const int *T, int nt,
                 const float *samples, int ns, double density) {
    if (w->n_assets == w->cap_assets) {
        w->cap_assets = w->cap_assets ? 2 * w->cap_assets : 4;
        w->assets = (asset_t *)realloc(w->assets, w->cap_assets * sizeof(asset_t));
    }
    asset_t *a = &w->assets[w->n_assets];
    memset(a, 0, sizeof *a);
    a->V = (float *)malloc(3 * sizeof(float) * nv); memcpy(a->V, V, 3 * sizeof(float) * nv);
    a->T = (int *)malloc(3 * sizeof(int) * nt); memcpy(a->T, T, 3 * sizeof(int) * nt);
    a->nv = nv; a->nt = nt;
    if (samples && ns > 0) {
        a->S = (float *)malloc(3 * sizeof(float) * ns); memcpy(a->S, samples, 3 * sizeof(float) * ns);
        a->ns = ns;
    }
    a->density = density;
    or_mass_properties(V, T, nt, density, &a->mass, a->com, a->I);
    double r2 = 0.0;
    for (int i = 0; i < nv; ++i) {
        const double x = V[3 * i], y = V[3 * i + 1], z = V[3 * i + 2];
        if (x * x + y * y + z * z > r2) r2 = x * x + y * y + z * z;
    }
    for (int i = 0; i < a->ns; ++i) {
        const double x = a->S[3 * i], y = a->S[3 * i + 1], z = a->S[3 * i + 2];
        if (x * x + y * y + z * z > r2) r2 = x * x + y * y + z * z;
    }
    a->radius = sqrt(r2);
    return w->n_assets++;
}

static void grid_alloc(grid_t *g, const float lo[3], float h, const int dims[3], int lazy) {
    for (int a = 0; a < 3; ++a) { g->lo[a] = lo[a]; g->dims[a] = dims[a]; }
    g->h = h;
    long long n = (long long)dims[0] * dims[1] * dims[2];
    free(g->val); free(g->done); free(g->bstate);
    g->val = (double *)calloc(n, sizeof(double));
    g->done = lazy ? (unsigned char *)calloc(n, 1) : NULL;
    g->lazy = lazy;
    g->bstate = NULL;
    g->band = 0.0f;
}

int or_asset_bake(or_world *w, int asset, int res, float pad, int cubic, int lazy) {
    asset_t *a = &w->assets[asset];
    float lo[3], h; int dims[3];
    or_grid_params(a->V, a->nv, res, pad, cubic, lo, &h, dims);
    grid_alloc(&a->grid, lo, h, dims, lazy);
    if (!lazy) or_bake_nodes(a->V, a->T, a->nt, lo, h, dims, NULL, 0, a->grid.val, w->cfg.n_threads);
    grid_set_band(&a->grid, w->cfg.sdf_band);
    a->has_grid = 1;
    return 0;
}

int or_asset_set_grid(or_world *w, int asset, const float lo[3], float h, const int dims[3],
                      const float *values) {
    asset_t *a = &w->assets[asset];
    grid_alloc(&a->grid, lo, h, dims, 0);
    long long n = (long long)dims[0] * dims[1] * dims[2];
    for (long long i = 0; i < n; ++i) a->grid.val[i] = values[i];
    grid_set_band(&a->grid, w->cfg.sdf_band);
    a->has_grid = 1;
    return 0;
}

int or_asset_get_grid(const or_world *w, int asset, float lo[3], float *h, int dims[3]) {
    const asset_t *a = &w->assets[asset];
    if (!a->has_grid) return -1;
    for (int i = 0; i < 3; ++i) { lo[i] = (float)a->grid.lo[i]; dims[i] = a->grid.dims[i]; }
    *h = (float)a->grid.h;
    return 0;
}

int or_asset_mass(const or_world *w, int asset, double *mass, double com[3], double inertia[9]) {
    const asset_t *a = &w->assets[asset];
    *mass = a->mass;
    memcpy(com, a->com, sizeof a->com);
    memcpy(inertia, a->I, sizeof a->I);
    return 0;
}

/* world inverse inertia and inertia of a body at its current orientation */
static void body_world_inertia(const body_t *b, double Iw[9], double Iw_inv[9]) {
    double R[9], Rt[9], tmp[9];
    q_to_m(b->q, R);
    m_transpose(R, Rt);
    if (b->type == 2 || b->type == 3) {
        m_mul(R, b->Ib, tmp); m_mul(tmp, Rt, Iw);
        if (b->type == 2) {
            m_mul(R, b->Ib_inv, tmp); m_mul(tmp, Rt, Iw_inv);
        } else {
            double Iaa = 0;
            double Ia[3];
            m_vec(Iw, b->axis, Ia);
            Iaa = v_dot(b->axis, Ia);
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) Iw_inv[3 * i + j] = b->axis[i] * b->axis[j] / Iaa;
        }
    } else {
        memset(Iw, 0, 9 * sizeof(double));
        memset(Iw_inv, 0, 9 * sizeof(double));
    }
}

static void body_com_world(const body_t *b, double c[3]) {
    double R[9];
    q_to_m(b->q, R);
    m_vec(R, b->com_b, c);
    v_add(c, b->p, c);
}

int or_add_envs(or_world *w, int n_envs, const or_body_desc *bd, int n_per_env,
                const int *pairs, int n_pairs) {
    const int pile = n_pairs < 0;   /* R20: pairs from the broad phase at every detection */
    if (pile) n_pairs = 0;
    int nb0 = w->n_bodies, np0 = w->n_pairs, ne0 = w->n_envs;
    w->bodies = (body_t *)realloc(w->bodies, sizeof(body_t) * (nb0 + n_envs * n_per_env));
    w->pairs = (pair_t *)realloc(w->pairs, sizeof(pair_t) * (np0 + n_envs * n_pairs));
    w->pc = (pair_contacts_t *)realloc(w->pc, sizeof(pair_contacts_t) * (np0 + n_envs * n_pairs));
    w->envs = (env_t *)realloc(w->envs, sizeof(env_t) * (ne0 + n_envs));
    w->env_mlen = (double *)realloc(w->env_mlen, sizeof(double) * (ne0 + n_envs));
    w->env_mdot = (double *)realloc(w->env_mdot, sizeof(double) * (ne0 + n_envs));
    w->imp = (double **)realloc(w->imp, sizeof(double *) * (ne0 + n_envs));
    w->imp_n = (int *)realloc(w->imp_n, sizeof(int) * (ne0 + n_envs));
    for (int e = 0; e < n_envs; ++e) { w->imp[ne0 + e] = NULL; w->imp_n[ne0 + e] = 0; }
    for (int e = 0; e < n_envs; ++e) {
        env_t *E = &w->envs[ne0 + e];
        E->first_body = nb0 + e * n_per_env;
        E->n_bodies = n_per_env;
        E->first_pair = np0 + e * n_pairs;
        E->n_pairs = n_pairs;
        E->pile = pile;
        E->dp = NULL; E->dpc = NULL; E->ndp = 0; E->cap_dp = 0;
        w->env_mlen[ne0 + e] = INFINITY;
        w->env_mdot[ne0 + e] = INFINITY;
        for (int i = 0; i < n_per_env; ++i) {
            const or_body_desc *d = &bd[e * n_per_env + i];
            body_t *b = &w->bodies[E->first_body + i];
            memset(b, 0, sizeof *b);
            const asset_t *A = &w->assets[d->asset];
            b->asset = d->asset; b->type = d->type; b->mu = d->mu;
            double scale = 1.0;
            b->mass = A->mass;
            if (d->mass > 0.0f) { scale = (double)d->mass / A->mass; b->mass = d->mass; }
            for (int k = 0; k < 9; ++k) b->Ib[k] = A->I[k] * scale;
            m_inverse(b->Ib, b->Ib_inv);
            memcpy(b->com_b, A->com, sizeof A->com);
            b->invm = (b->type == 2) ? 1.0 / b->mass : 0.0;
            load3(d->axis, b->axis);
            double an = v_norm(b->axis);
            if (an > 0) v_scale(b->axis, 1.0 / an, b->axis);
            load3(d->force, b->force); load3(d->torque, b->torque);
            load3(d->pos, b->p);
            for (int k = 0; k < 4; ++k) b->q[k] = d->quat[k];
            q_normalize(b->q);
            /* linvel / angvel are of the centre of mass; fixed-axis bodies keep the
               centre fixed and spin about the axis only */
            load3(d->linvel, b->v); load3(d->angvel, b->w);
            if (b->type == 0) { memset(b->v, 0, sizeof b->v); memset(b->w, 0, sizeof b->w); }
            if (b->type == 3) { double s = v_dot(b->w, b->axis); memset(b->v, 0, sizeof b->v); v_scale(b->axis, s, b->w); }
        }
        for (int p = 0; p < n_pairs; ++p) {
            pair_t *P = &w->pairs[E->first_pair + p];
            P->a = E->first_body + pairs[2 * p];
            P->b = E->first_body + pairs[2 * p + 1];
            P->mu = sqrt((double)w->bodies[P->a].mu * (double)w->bodies[P->b].mu);
            P->color = 0;
            pair_contacts_t *pc = &w->pc[E->first_pair + p];
            memset(pc, 0, sizeof *pc);
            pc->m_len = INFINITY; pc->m_dot = INFINITY;
        }
    }
    w->n_bodies = nb0 + n_envs * n_per_env;
    w->n_pairs = np0 + n_envs * n_pairs;
    w->n_envs = ne0 + n_envs;
    return ne0;
}

int or_n_envs(const or_world *w) { return w->n_envs; }
int or_n_bodies(const or_world *w) { return w->n_bodies; }

/* ------------------------------------------------------------------------------------ */
/* Algorithm 1 (Sec. III-C)                                                               */
/* ------------------------------------------------------------------------------------ */
typedef struct { int idx; double phi, x[3], n[3]; } cand_t;

#define NSLOT 7
typedef struct {
    double n[3], a[3], t1[3], t2[3];
    int idx[NSLOT];
    double best[NSLOT], second[NSLOT];
    cand_t mem[NSLOT];
} patch_t;

typedef struct { double len, dot; } margin_t;

static void mark_len(margin_t *m, double v) { v = fabs(v); if (v < m->len) m->len = v; }
static void mark_dot(margin_t *m, double v) { v = fabs(v); if (v < m->dot) m->dot = v; }

/* R11 */
static void tangent_basis(const double n[3], double t1[3], double t2[3], margin_t *m) {
    static const double ex[3] = {1, 0, 0}, ey[3] = {0, 1, 0};
    if (m) mark_dot(m, fabs(n[0]) - 0.57735);
    if (fabs(n[0]) < 0.57735) v_cross(n, ex, t1); else v_cross(n, ey, t1);
    v_scale(t1, 1.0 / v_norm(t1), t1);
    v_cross(n, t1, t2);
}

static double slot_score(const patch_t *P, const cand_t *c, int s) {
    if (s == 0) return -c->phi;                         /* deepest */
    double ang = (double)(s - 1) * M_PI / 3.0;
    double u[3], d[3];
    for (int i = 0; i < 3; ++i) u[i] = cos(ang) * P->t1[i] + sin(ang) * P->t2[i];
    v_sub(c->x, P->a, d);
    return v_dot(d, u);
}

static void patch_init(patch_t *P, const cand_t *seed, margin_t *m) {
    memcpy(P->n, seed->n, sizeof P->n);
    memcpy(P->a, seed->x, sizeof P->a);
    tangent_basis(P->n, P->t1, P->t2, m);
    for (int s = 0; s < NSLOT; ++s) { P->idx[s] = -1; P->best[s] = -INFINITY; P->second[s] = -INFINITY; }
}

/* running argmax per slot, ties to the lowest sample index; margin = best - second */
static void patch_add_member(patch_t *P, const cand_t *c) {
    for (int s = 0; s < NSLOT; ++s) {
        double v = slot_score(P, c, s);
        if (P->idx[s] < 0 || v > P->best[s] || (v == P->best[s] && c->idx < P->idx[s])) {
            P->second[s] = P->best[s];
            P->best[s] = v; P->idx[s] = c->idx; P->mem[s] = *c;
        } else if (v > P->second[s]) {
            P->second[s] = v;
        }
    }
}

static void patch_slot_margins(const patch_t *P, margin_t *m, int exact_phi) {
    for (int s = exact_phi ? 1 : 0; s < NSLOT; ++s)
        if (P->idx[s] >= 0 && P->second[s] > -INFINITY) mark_len(m, P->best[s] - P->second[s]);
}

/* R8: M = -phi_deepest + sqrt(area of the polygon through the distinct direction-slot
 * points, in slot order, in the (t1, t2) plane) */
static double patch_measure(const patch_t *P) {
    double xs[6], ys[6];
    int n = 0, seen[6];
    for (int s = 1; s < NSLOT; ++s) {
        int dup = 0;
        if (P->idx[s] < 0) continue;
        for (int t = 0; t < n; ++t) if (seen[t] == P->idx[s]) dup = 1;
        if (dup) continue;
        double d[3];
        v_sub(P->mem[s].x, P->a, d);
        xs[n] = v_dot(d, P->t1); ys[n] = v_dot(d, P->t2);
        seen[n++] = P->idx[s];
    }
    double area2 = 0.0;
    for (int i = 0; i < n; ++i) {
        int j = (i + 1) % n;
        area2 += xs[i] * ys[j] - xs[j] * ys[i];
    }
    double area = 0.5 * fabs(area2);
    return -P->mem[0].phi + sqrt(area);
}

typedef struct {
    patch_t *p; int n, cap;
} patch_list_t;

/* AddPatch (Sec. III-C): append below capacity, else replace the most similar patch
 * if the new one scores higher on M, else drop it */
static void add_patch(patch_list_t *L, const patch_t *P, int max_patches, margin_t *m) {
    if (L->n < max_patches) { L->p[L->n++] = *P; return; }
    int k = 0; double bd = -INFINITY, sd = -INFINITY;
    for (int j = 0; j < L->n; ++j) {
        double d = v_dot(P->n, L->p[j].n);
        if (d > bd) { sd = bd; bd = d; k = j; } else if (d > sd) sd = d;
    }
    if (sd > -INFINITY) mark_dot(m, bd - sd);
    double mn = patch_measure(P), mo = patch_measure(&L->p[k]);
    mark_len(m, mn - mo);
    if (mn > mo) L->p[k] = *P;
}

/* Algorithm 1 over one shape pair.  cands must be sorted by sample index. */
/* exact_phi = 1 when both sides compare the very same phi values (float inputs): the
 * decisions that compare phi only (FindDeepest, the deepest slot) then cannot differ and
 * are not counted as margins. */
static int reduce_pair(const cand_t *cands, int nc, double cos_patch, int max_patches,
                       int batch_size, or_contact *out, int cap, int *n_patches, margin_t *m,
                       int exact_phi) {
    patch_list_t L;
    L.cap = max_patches; L.n = 0;
    L.p = (patch_t *)malloc(sizeof(patch_t) * (max_patches > 0 ? max_patches : 1));
    int *assigned = (int *)malloc(sizeof(int) * (nc > 0 ? nc : 1));
    int start = 0;
    while (start < nc) {
        /* Generate: the candidates of this batch of samples */
        int bidx = cands[start].idx / batch_size, end = start;
        while (end < nc && cands[end].idx / batch_size == bidx) ++end;
        /* Assign to existing patches by normal similarity */
        int n_existing = L.n;
        for (int i = start; i < end; ++i) {
            assigned[i] = 0;
            int best = -1; double bd = -INFINITY, sd = -INFINITY;
            for (int j = 0; j < n_existing; ++j) {
                double d = v_dot(cands[i].n, L.p[j].n);
                if (d > bd) { sd = bd; bd = d; best = j; } else if (d > sd) sd = d;
            }
            if (best < 0) continue;
            mark_dot(m, bd - cos_patch);
            if (bd >= cos_patch) {
                if (sd > -INFINITY) mark_dot(m, bd - sd);
                patch_add_member(&L.p[best], &cands[i]);
                assigned[i] = 1;
            }
        }
        /* while candidates remain: FindDeepest, BinReduce, AddPatch */
        for (;;) {
            int best = -1; double bphi = INFINITY, sphi = INFINITY;
            for (int i = start; i < end; ++i) {
                if (assigned[i]) continue;
                /* candidates are visited in sample order, so '<' keeps the lowest index on ties */
                if (cands[i].phi < bphi) {
                    sphi = bphi; bphi = cands[i].phi; best = i;
                } else if (cands[i].phi < sphi) sphi = cands[i].phi;
            }
            if (best < 0) break;
            if (sphi < INFINITY && !exact_phi) mark_len(m, sphi - bphi);
            patch_t P;
            patch_init(&P, &cands[best], m);
            for (int i = start; i < end; ++i) {
                if (assigned[i]) continue;
                double d = v_dot(cands[i].n, P.n);
                if (i != best) mark_dot(m, d - cos_patch);
                if (i == best || d >= cos_patch) {
                    patch_add_member(&P, &cands[i]);
                    assigned[i] = 1;
                }
            }
            add_patch(&L, &P, max_patches, m);
        }
        start = end;
    }
    /* emit: patches in list order, distinct slot members in slot order */
    int n = 0;
    for (int j = 0; j < L.n; ++j) {
        patch_slot_margins(&L.p[j], m, exact_phi);
        for (int s = 0; s < NSLOT; ++s) {
            int id = L.p[j].idx[s], dup = 0;
            if (id < 0) continue;
            for (int t = 0; t < s; ++t) if (L.p[j].idx[t] == id) dup = 1;
            if (dup) continue;
            if (n < cap) {
                const cand_t *c = &L.p[j].mem[s];
                or_contact *o = &out[n];
                o->sample = c->idx; o->patch = j; o->phi = c->phi;
                for (int a = 0; a < 3; ++a) {
                    o->xa[a] = c->x[a]; o->n[a] = c->n[a];
                    o->xb[a] = c->x[a] - c->phi * c->n[a];
                }
            }
            ++n;
        }
    }
    *n_patches = L.n;
    free(L.p); free(assigned);
    return n;
}

int or_reduce(const or_candidate *cand, int n, double cos_patch, int max_patches,
              int batch_size, or_contact *out, int cap, int *n_out, int *n_patches,
              double *min_margin_len, double *min_margin_dot) {
    cand_t *c = (cand_t *)malloc(sizeof(cand_t) * (n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        c[i].idx = cand[i].sample; c[i].phi = cand[i].phi;
        load3(cand[i].x, c[i].x); load3(cand[i].n, c[i].n);
    }
    /* insertion into sample order (stable) */
    for (int i = 1; i < n; ++i) {
        cand_t t = c[i]; int j = i - 1;
        while (j >= 0 && c[j].idx > t.idx) { c[j + 1] = c[j]; --j; }
        c[j + 1] = t;
    }
    margin_t m = {INFINITY, INFINITY};
    int np = 0;
    int k = reduce_pair(c, n, cos_patch, max_patches, batch_size, out, cap, &np, &m, 1);
    *n_out = k; *n_patches = np;
    *min_margin_len = m.len; *min_margin_dot = m.dot;
    free(c);
    return k > cap ? -1 : 0;
}

/* ------------------------------------------------------------------------------------ */
/* narrow phase of one pair at the current poses (Sec. III-A; R4, R5)                    */
/* ------------------------------------------------------------------------------------ */
static void ensure_nodes(or_world *w);

/* R15: local minimisation of phi over the face (a, b, c), all in the SDF's frame.
 * Returns 1 with the minimiser x, phi and gradient there; 0 when the centroid is outside
 * the grid.  *margin: smallest |phi_trial - phi| over the step decisions. */
static int tri_minimise(const grid_t *g, const double a[3], const double b[3], const double c[3], int iters,
                        double x[3], double *phi, double grad[3], double *margin) {
    double e1[3], e2[3], e3[3], nt[3];
    v_sub(b, a, e1); v_sub(c, a, e2); v_sub(c, b, e3);
    v_cross(e1, e2, nt);
    double ntn = v_norm(nt);
    for (int k = 0; k < 3; ++k) x[k] = (a[k] + b[k] + c[k]) / 3.0;
    *margin = INFINITY;
    if (!trilinear(g, x, phi, grad, NULL)) return 0;
    if (ntn > 0.0) v_scale(nt, 1.0 / ntn, nt);
    double s = 0.5 * fmax(v_norm(e1), fmax(v_norm(e2), v_norm(e3)));
    for (int it = 0; it < iters; ++it) {
        /* the gradient's part in the face's plane */
        double d[3], gn = v_dot(grad, nt);
        for (int k = 0; k < 3; ++k) d[k] = grad[k] - gn * nt[k];
        double dn = v_norm(d);
        if (!(dn > 1e-9)) break;
        double p[3], xt[3], pt, gt[3];
        for (int k = 0; k < 3; ++k) p[k] = x[k] - (s / dn) * d[k];
        or_closest_point_triangle(p, a, b, c, xt);
        int ok = trilinear(g, xt, &pt, gt, NULL);
        if (ok && fabs(pt - *phi) < *margin) *margin = fabs(pt - *phi);
        if (ok && pt < *phi) {
            memcpy(x, xt, sizeof xt); *phi = pt; memcpy(grad, gt, sizeof gt);
            s *= 1.5;
        } else {
            s *= 0.5;
        }
    }
    return 1;
}

/* the face of body a's mesh, in body b's (SDF) frame */
static void tri_in_b(const asset_t *aa, int t, const double RA[9], const double pA[3], const double RBt[9],
                     const double pB[3], double v[3][3]) {
    for (int k = 0; k < 3; ++k) {
        double s[3], xw[3], d[3];
        load3(aa->V + 3 * aa->T[3 * t + k], s);
        m_vec(RA, s, xw); v_add(xw, pA, xw);
        v_sub(xw, pB, d); m_vec(RBt, d, v[k]);
    }
}

static int generate_tri_candidates(const or_world *w, const pair_t *P, cand_t *out, margin_t *m) {
    const body_t *A = &w->bodies[P->a], *B = &w->bodies[P->b];
    const asset_t *aa = &w->assets[A->asset], *ab = &w->assets[B->asset];
    double RA[9], RB[9], RBt[9];
    q_to_m(A->q, RA); q_to_m(B->q, RB); m_transpose(RB, RBt);
    int n = 0;
    for (int t = 0; t < aa->nt; ++t) {
        double v[3][3], x[3], phi, g[3], mg;
        tri_in_b(aa, t, RA, A->p, RBt, B->p, v);
        if (!tri_minimise(&ab->grid, v[0], v[1], v[2], w->cfg.tri_iters, x, &phi, g, &mg)) continue;
        mark_len(m, mg);
        double gn = v_norm(g);
        if (gn < 1e-12) continue;
        mark_len(m, phi - w->cfg.contact_offset);
        if (!(phi < w->cfg.contact_offset)) continue;
        double nb[3];
        v_scale(g, 1.0 / gn, nb);
        cand_t *c = &out[n++];
        c->idx = t; c->phi = phi;
        m_vec(RB, x, c->x); v_add(c->x, B->p, c->x);
        m_vec(RB, nb, c->n);
    }
    return n;
}

static int generate_candidates(const or_world *w, const pair_t *P, cand_t *out, margin_t *m) {
    if (w->cfg.contact_gen == 1) return generate_tri_candidates(w, P, out, m);
    const body_t *A = &w->bodies[P->a], *B = &w->bodies[P->b];
    const asset_t *aa = &w->assets[A->asset], *ab = &w->assets[B->asset];
    double RA[9], RB[9], RBt[9];
    q_to_m(A->q, RA); q_to_m(B->q, RB); m_transpose(RB, RBt);
    int n = 0;
    for (int i = 0; i < aa->ns; ++i) {
        double s[3], xw[3], xb[3], d[3], phi, g[3], bm;
        load3(aa->S + 3 * i, s);
        m_vec(RA, s, xw); v_add(xw, A->p, xw);
        v_sub(xw, B->p, d); m_vec(RBt, d, xb);
        int ok = trilinear(&ab->grid, xb, &phi, g, &bm);
        mark_len(m, bm);
        if (!ok) continue;
        double gn = v_norm(g);
        if (gn < 1e-12) continue;
        mark_len(m, phi - w->cfg.contact_offset);
        if (!(phi < w->cfg.contact_offset)) continue;
        double nb[3];
        v_scale(g, 1.0 / gn, nb);
        cand_t *c = &out[n++];
        c->idx = i; c->phi = phi;
        memcpy(c->x, xw, sizeof xw);
        m_vec(RB, nb, c->n);
    }
    return n;
}

/* The pairs of an env and their contacts: the listed pairs, or a pile's current list. */
static pair_t *env_pairs(const or_world *w, int e) {
    const env_t *E = &w->envs[e];
    return E->pile ? E->dp : &w->pairs[E->first_pair];
}
static pair_contacts_t *env_pcs(const or_world *w, int e) {
    const env_t *E = &w->envs[e];
    return E->pile ? E->dpc : &w->pc[E->first_pair];
}
static int env_np(const or_world *w, int e) {
    const env_t *E = &w->envs[e];
    return E->pile ? E->ndp : E->n_pairs;
}

static int movable(const body_t *b) { return b->type == 2 || b->type == 3; }

/* R20: the pairs of a pile env, rebuilt at every detection.  For bodies i < j (env order),
 * at least one of them movable: body i's samples against body j's SDF when i has samples
 * and j a grid, else body j's samples against body i's SDF when j has samples and i a grid,
 * else no pair.  A pair whose bounding spheres (about the asset origins) are farther apart
 * than the contact offset plus two voxels of the SDF body is left out: no sample can have
 * a candidate there (R19), so leaving it out changes no contact.  Pairs in (i, j) order. */
static void pile_pairs(or_world *w, int e) {
    env_t *E = &w->envs[e];
    int n = 0;
    for (int i = 0; i < E->n_bodies; ++i)
        for (int j = i + 1; j < E->n_bodies; ++j) {
            const body_t *Bi = &w->bodies[E->first_body + i], *Bj = &w->bodies[E->first_body + j];
            if (!movable(Bi) && !movable(Bj)) continue;
            const asset_t *Ai = &w->assets[Bi->asset], *Aj = &w->assets[Bj->asset];
            int a, b;
            if (Ai->ns > 0 && Aj->has_grid) { a = i; b = j; }
            else if (Aj->ns > 0 && Ai->has_grid) { a = j; b = i; }
            else continue;
            const body_t *BA = &w->bodies[E->first_body + a], *BB = &w->bodies[E->first_body + b];
            const asset_t *AA = &w->assets[BA->asset], *AB = &w->assets[BB->asset];
            double d[3];
            v_sub(BA->p, BB->p, d);
            const double lim = AA->radius + AB->radius + w->cfg.contact_offset + 2.0 * AB->grid.h;
            if (v_dot(d, d) > lim * lim) continue;
            if (n == E->cap_dp) {
                const int cap = E->cap_dp ? 2 * E->cap_dp : 64;
                E->dp = (pair_t *)realloc(E->dp, sizeof(pair_t) * cap);
                E->dpc = (pair_contacts_t *)realloc(E->dpc, sizeof(pair_contacts_t) * cap);
                memset(E->dpc + E->cap_dp, 0, sizeof(pair_contacts_t) * (cap - E->cap_dp));
                E->cap_dp = cap;
            }
            pair_t *P = &E->dp[n];
            P->a = E->first_body + a;
            P->b = E->first_body + b;
            P->mu = sqrt((double)BA->mu * (double)BB->mu);
            E->dpc[n].n = 0;
            E->dpc[n].m_len = INFINITY; E->dpc[n].m_dot = INFINITY;
            ++n;
        }
    E->ndp = n;
}

static void detect_pair(or_world *w, const pair_t *P, pair_contacts_t *pc) {
    const asset_t *aa = &w->assets[w->bodies[P->a].asset];
    const int n_src = w->cfg.contact_gen == 1 ? aa->nt : aa->ns;
    cand_t *c = (cand_t *)malloc(sizeof(cand_t) * (n_src > 0 ? n_src : 1));
    margin_t m = {INFINITY, INFINITY};
    int nc = generate_candidates(w, P, c, &m);
    int cap = w->cfg.max_patches * NSLOT;
    if (pc->cap < cap) { pc->c = (or_contact *)realloc(pc->c, sizeof(or_contact) * cap); pc->cap = cap; }
    pc->n = reduce_pair(c, nc, w->cfg.cos_patch, w->cfg.max_patches, w->cfg.batch_size,
                        pc->c, pc->cap, &pc->n_patches, &m, 0);
    pc->m_len = m.len; pc->m_dot = m.dot;
    free(c);
}

/* lazy bake: queue the nodes a lookup in cell c reads -- its 8 corners, or with bricked
 * storage (R17) every node of its brick, which the brick's state depends on */
static void queue_cell(grid_t *g, const int c[3], long long **need, long long *nn, long long *cap) {
    int n0[3], n1[3];
    for (int a = 0; a < 3; ++a) {
        if (g->band > 0.0f) {
            n0[a] = (c[a] / BRICK) * BRICK;
            n1[a] = n0[a] + BRICK;
            if (n1[a] > g->dims[a] - 1) n1[a] = g->dims[a] - 1;
        } else {
            n0[a] = c[a];
            n1[a] = c[a] + 1;
        }
    }
    if (g->band > 0.0f && g->bstate[brick_index(g, c[0], c[1], c[2])] != BRICK_UNKNOWN) return;
    for (int k = n0[2]; k <= n1[2]; ++k)
        for (int j = n0[1]; j <= n1[1]; ++j)
            for (int i = n0[0]; i <= n1[0]; ++i) {
                const long long id = gidx(g, i, j, k);
                if (g->done[id]) continue;
                g->done[id] = 2;    /* queued */
                if (*nn == *cap) { *cap *= 2; *need = (long long *)realloc(*need, sizeof(long long) * *cap); }
                (*need)[(*nn)++] = id;
            }
}

/* lazy bake: compute every grid node the next detection will read */
static double wall_seconds(void) {
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

static void ensure_nodes(or_world *w) {
    const double t0 = wall_seconds();
    for (int ai = 0; ai < w->n_assets; ++ai) {
        asset_t *ab = &w->assets[ai];
        if (!ab->has_grid || !ab->grid.lazy) continue;
        grid_t *g = &ab->grid;
        long long cap = 1024, nn = 0;
        long long *need = (long long *)malloc(sizeof(long long) * cap);
        int n_all = w->n_pairs;
        for (int e = 0; e < w->n_envs; ++e) n_all += w->envs[e].pile ? w->envs[e].ndp : 0;
        for (int pi = 0; pi < n_all; ++pi) {
            const pair_t *P = NULL;
            if (pi < w->n_pairs) P = &w->pairs[pi];
            else {   /* the pile envs' current pairs, env after env */
                int k = pi - w->n_pairs;
                for (int e = 0; e < w->n_envs && !P; ++e) {
                    if (!w->envs[e].pile) continue;
                    if (k < w->envs[e].ndp) P = &w->envs[e].dp[k];
                    else k -= w->envs[e].ndp;
                }
            }
            const body_t *A = &w->bodies[P->a], *B = &w->bodies[P->b];
            if (B->asset != ai) continue;
            const asset_t *aa = &w->assets[A->asset];
            double RA[9], RB[9], RBt[9];
            q_to_m(A->q, RA); q_to_m(B->q, RB); m_transpose(RB, RBt);
            if (w->cfg.contact_gen == 1) {   /* every cell a face's bounding box touches */
                for (int t = 0; t < aa->nt; ++t) {
                    double v[3][3];
                    tri_in_b(aa, t, RA, A->p, RBt, B->p, v);
                    int c0[3], c1[3];
                    for (int a = 0; a < 3; ++a) {
                        double lo = fmin(v[0][a], fmin(v[1][a], v[2][a])), hi = fmax(v[0][a], fmax(v[1][a], v[2][a]));
                        c0[a] = (int)floor((lo - g->lo[a]) / g->h); c1[a] = (int)floor((hi - g->lo[a]) / g->h);
                        if (c0[a] < 0) c0[a] = 0;
                        if (c1[a] > g->dims[a] - 2) c1[a] = g->dims[a] - 2;
                    }
                    for (int k = c0[2]; k <= c1[2]; ++k)
                        for (int j = c0[1]; j <= c1[1]; ++j)
                            for (int i = c0[0]; i <= c1[0]; ++i) {
                                const int c[3] = {i, j, k};
                                queue_cell(g, c, &need, &nn, &cap);
                            }
                }
                continue;
            }
            for (int i = 0; i < aa->ns; ++i) {
                double s[3], xw[3], xb[3], d[3];
                load3(aa->S + 3 * i, s);
                m_vec(RA, s, xw); v_add(xw, A->p, xw);
                v_sub(xw, B->p, d); m_vec(RBt, d, xb);
                int c[3], inside = 1;
                for (int a = 0; a < 3; ++a) {
                    double u = (xb[a] - g->lo[a]) / g->h;
                    if (!(u >= 0.0 && u <= g->dims[a] - 1)) inside = 0;
                    int ci = (int)floor(u);
                    if (ci > g->dims[a] - 2) ci = g->dims[a] - 2;
                    if (ci < 0) ci = 0;
                    c[a] = ci;
                }
                if (!inside) continue;
                queue_cell(g, c, &need, &nn, &cap);
            }
        }
        if (nn > 0) {
            double *vals = (double *)malloc(sizeof(double) * nn);
            float lo[3] = {(float)g->lo[0], (float)g->lo[1], (float)g->lo[2]};
            or_bake_nodes(ab->V, ab->T, ab->nt, lo, (float)g->h, g->dims, need, nn, vals, w->cfg.n_threads);
            for (long long q = 0; q < nn; ++q) { g->val[need[q]] = vals[q]; g->done[need[q]] = 1; }
            free(vals);
        }
        free(need);
        if (g->band > 0.0f)   /* R17: states of the bricks whose nodes are now all baked */
            for (int bk = 0; bk < g->bdims[2]; ++bk)
                for (int bj = 0; bj < g->bdims[1]; ++bj)
                    for (int bi = 0; bi < g->bdims[0]; ++bi) {
                        signed char *st = &g->bstate[brick_index(g, bi * BRICK, bj * BRICK, bk * BRICK)];
                        if (*st == BRICK_UNKNOWN) *st = brick_state(g, bi, bj, bk);
                    }
    }
    w->bake_seconds += wall_seconds() - t0;
}

double or_bake_seconds(const or_world *w) { return w->bake_seconds; }

/* narrow phase of one pair, every sample: phi and world normal (valid = 0 where the
 * sample is outside the grid or the gradient vanishes) */
int or_query_pair(or_world *w, int env, int pair, double *phi, double *nrm, int *valid, double *gnorm) {
    ensure_nodes(w);
    const pair_t *P = &env_pairs(w, env)[pair];
    const body_t *A = &w->bodies[P->a], *B = &w->bodies[P->b];
    const asset_t *aa = &w->assets[A->asset], *ab = &w->assets[B->asset];
    double RA[9], RB[9], RBt[9];
    q_to_m(A->q, RA); q_to_m(B->q, RB); m_transpose(RB, RBt);
    for (int i = 0; i < aa->ns; ++i) {
        double s[3], xw[3], xb[3], d[3], g[3], f;
        load3(aa->S + 3 * i, s);
        m_vec(RA, s, xw); v_add(xw, A->p, xw);
        v_sub(xw, B->p, d); m_vec(RBt, d, xb);
        int ok = trilinear(&ab->grid, xb, &f, g, NULL);
        double gn = ok ? v_norm(g) : 0.0;
        valid[i] = ok && gn >= 1e-12;
        phi[i] = valid[i] ? f : 0.0;
        if (gnorm) gnorm[i] = gn;
        for (int a = 0; a < 3; ++a) nrm[3 * i + a] = 0.0;
        if (valid[i]) {
            double nb[3];
            v_scale(g, 1.0 / gn, nb);
            m_vec(RB, nb, nrm + 3 * i);
        }
    }
    return 0;
}

/* the candidates of one pair (Generate of Algorithm 1), rounded to float */
int or_pair_candidates(or_world *w, int env, int pair, or_candidate *out, int cap, int *n_out) {
    ensure_nodes(w);
    const pair_t *P = &env_pairs(w, env)[pair];
    const asset_t *aa = &w->assets[w->bodies[P->a].asset];
    const int n_src = w->cfg.contact_gen == 1 ? aa->nt : aa->ns;
    cand_t *c = (cand_t *)malloc(sizeof(cand_t) * (n_src > 0 ? n_src : 1));
    margin_t m = {INFINITY, INFINITY};
    int n = generate_candidates(w, P, c, &m);
    for (int i = 0; i < n && i < cap; ++i) {
        out[i].sample = c[i].idx;
        out[i].phi = (float)c[i].phi;
        for (int a = 0; a < 3; ++a) { out[i].x[a] = (float)c[i].x[a]; out[i].n[a] = (float)c[i].n[a]; }
    }
    *n_out = n;
    free(c);
    return n > cap ? -1 : 0;
}

int or_tri_contacts(or_world *w, int env, int pair, double *x, double *phi, double *n, int *valid,
                    double *margin) {
    ensure_nodes(w);
    const pair_t *P = &env_pairs(w, env)[pair];
    const body_t *A = &w->bodies[P->a], *B = &w->bodies[P->b];
    const asset_t *aa = &w->assets[A->asset], *ab = &w->assets[B->asset];
    double RA[9], RB[9], RBt[9];
    q_to_m(A->q, RA); q_to_m(B->q, RB); m_transpose(RB, RBt);
    for (int t = 0; t < aa->nt; ++t) {
        double v[3][3], xb[3], p, g[3], mg;
        tri_in_b(aa, t, RA, A->p, RBt, B->p, v);
        int ok = tri_minimise(&ab->grid, v[0], v[1], v[2], w->cfg.tri_iters, xb, &p, g, &mg);
        double gn = ok ? v_norm(g) : 0.0;
        valid[t] = ok && gn >= 1e-12;
        phi[t] = ok ? p : 0.0;
        margin[t] = mg;
        m_vec(RB, xb, x + 3 * t); v_add(x + 3 * t, B->p, x + 3 * t);
        double nb[3] = {0, 0, 0};
        if (valid[t]) v_scale(g, 1.0 / gn, nb);
        m_vec(RB, nb, n + 3 * t);
    }
    return 0;
}

int or_collide(or_world *w) {
    for (int e = 0; e < w->n_envs; ++e)
        if (w->envs[e].pile) pile_pairs(w, e);
    ensure_nodes(w);
    int n_all = w->n_pairs;
    for (int e = 0; e < w->n_envs; ++e) n_all += w->envs[e].pile ? w->envs[e].ndp : 0;
    const pair_t **lp = (const pair_t **)malloc(sizeof(pair_t *) * (n_all > 0 ? n_all : 1));
    pair_contacts_t **lc = (pair_contacts_t **)malloc(sizeof(pair_contacts_t *) * (n_all > 0 ? n_all : 1));
    int k = 0;
    for (int pi = 0; pi < w->n_pairs; ++pi, ++k) { lp[k] = &w->pairs[pi]; lc[k] = &w->pc[pi]; }
    for (int e = 0; e < w->n_envs; ++e)
        if (w->envs[e].pile)
            for (int p = 0; p < w->envs[e].ndp; ++p, ++k) { lp[k] = &w->envs[e].dp[p]; lc[k] = &w->envs[e].dpc[p]; }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(team_size(w->cfg.n_threads))
#endif
    for (int q = 0; q < n_all; ++q) detect_pair(w, lp[q], lc[q]);
    free(lp); free(lc);
    for (int e = 0; e < w->n_envs; ++e) {
        const pair_contacts_t *pcs = env_pcs(w, e);
        for (int p = 0; p < env_np(w, e); ++p) {
            const pair_contacts_t *pc = &pcs[p];
            if (pc->m_len < w->env_mlen[e]) w->env_mlen[e] = pc->m_len;
            if (pc->m_dot < w->env_mdot[e]) w->env_mdot[e] = pc->m_dot;
        }
    }
    return 0;
}

int or_get_contacts(const or_world *w, int env, or_contact *out, int cap, int *n_out,
                    double *min_margin_len, double *min_margin_dot) {
    int n = 0;
    double ml = INFINITY, md = INFINITY;
    const pair_contacts_t *pcs = env_pcs(w, env);
    for (int p = 0; p < env_np(w, env); ++p) {
        const pair_contacts_t *pc = &pcs[p];
        for (int i = 0; i < pc->n; ++i) {
            if (n < cap) out[n] = pc->c[i];
            ++n;
        }
        if (pc->m_len < ml) ml = pc->m_len;
        if (pc->m_dot < md) md = pc->m_dot;
    }
    *n_out = n;
    if (min_margin_len) *min_margin_len = ml;
    if (min_margin_dot) *min_margin_dot = md;
    return n > cap ? -1 : 0;
}

/* contacts of an env go to its first pair (the solve only needs them in order); a pile
 * env's contacts are set pair by pair (or_set_pair_contacts) */
int or_set_contacts(or_world *w, int env, const or_contact *in, int n) {
    const env_t *E = &w->envs[env];
    if (E->pile) return -1;
    for (int p = 0; p < E->n_pairs; ++p) w->pc[E->first_pair + p].n = 0;
    pair_contacts_t *pc = &w->pc[E->first_pair];
    if (pc->cap < n) { pc->c = (or_contact *)realloc(pc->c, sizeof(or_contact) * n); pc->cap = n; }
    memcpy(pc->c, in, sizeof(or_contact) * n);
    pc->n = n;
    return 0;
}

int or_get_pair_contacts(const or_world *w, int env, int pair, or_contact *out, int cap, int *n_out) {
    if (env < 0 || env >= w->n_envs || pair < 0 || pair >= env_np(w, env)) return -1;
    const pair_contacts_t *pc = &env_pcs(w, env)[pair];
    for (int i = 0; i < pc->n && i < cap; ++i) out[i] = pc->c[i];
    *n_out = pc->n;
    return pc->n > cap ? -1 : 0;
}

int or_set_pair_contacts(or_world *w, int env, int pair, const or_contact *in, int n) {
    if (env < 0 || env >= w->n_envs || pair < 0 || pair >= env_np(w, env) || n < 0) return -1;
    pair_contacts_t *pc = &env_pcs(w, env)[pair];
    if (pc->cap < n) { pc->c = (or_contact *)realloc(pc->c, sizeof(or_contact) * (n > 0 ? n : 1)); pc->cap = n; }
    if (n > 0) memcpy(pc->c, in, sizeof(or_contact) * n);
    pc->n = n;
    return 0;
}

/* A pile env's current pairs (from its last detection): (point body, SDF body) as local
 * body ids, in pair order; the pair's colour in the last solve (-1: no contacts). */
int or_get_pile_pairs(const or_world *w, int env, int *ab, int *color, int cap, int *n_out) {
    if (env < 0 || env >= w->n_envs || !w->envs[env].pile) return -1;
    const env_t *E = &w->envs[env];
    for (int p = 0; p < E->ndp && p < cap; ++p) {
        ab[2 * p] = E->dp[p].a - E->first_body;
        ab[2 * p + 1] = E->dp[p].b - E->first_body;
        if (color) color[p] = E->dp[p].color;
    }
    *n_out = E->ndp;
    return E->ndp > cap ? -1 : 0;
}

/* The smallest decision margins of one pair's last detection. */
int or_pair_margins(const or_world *w, int env, int pair, double *len, double *dot) {
    if (env < 0 || env >= w->n_envs || pair < 0 || pair >= env_np(w, env)) return -1;
    const pair_contacts_t *pc = &env_pcs(w, env)[pair];
    *len = pc->m_len; *dot = pc->m_dot;
    return 0;
}

/* A pile env's pair list at the current poses, without detecting their contacts (the
 * broad phase alone; the pairs' contacts are cleared). */
int or_find_pile_pairs(or_world *w, int env) {
    if (env < 0 || env >= w->n_envs || !w->envs[env].pile) return -1;
    pile_pairs(w, env);
    return 0;
}

int or_env_margins(const or_world *w, int env, double *len, double *dot) {
    *len = w->env_mlen[env]; *dot = w->env_mdot[env];
    return 0;
}

void or_reset_margins(or_world *w) {
    for (int e = 0; e < w->n_envs; ++e) { w->env_mlen[e] = INFINITY; w->env_mdot[e] = INFINITY; }
}

/* ------------------------------------------------------------------------------------ */
/* substep (R9, R10)                                                                      */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    int a, b;                     /* local body index in the env */
    double ra[3], rb[3], n[3], t1[3], t2[3];
    double kn, kt1, kt2, bias, mu;
    double ln, lt1, lt2;
} row_t;

/* effective mass of direction d at the contact: 1 / (J M^-1 J^T) */
static double eff_mass(const body_t *A, const body_t *B, const double IA[9], const double IB[9],
                       const double ra[3], const double rb[3], const double d[3]) {
    double ca[3], cb[3], ta[3], tb[3];
    v_cross(ra, d, ca); v_cross(rb, d, cb);
    m_vec(IA, ca, ta); m_vec(IB, cb, tb);
    double den = A->invm + B->invm + v_dot(ca, ta) + v_dot(cb, tb);
    return den > 0.0 ? 1.0 / den : 0.0;
}

/* apply impulse p (world vector) at the contact: +p on A, -p on B */
static void apply_impulse(body_t *A, body_t *B, const double IA[9], const double IB[9],
                          const double ra[3], const double rb[3], const double p[3]) {
    double c[3], dw[3];
    v_axpy(A->invm, p, A->v);
    v_cross(ra, p, c); m_vec(IA, c, dw); v_add(A->w, dw, A->w);
    v_axpy(-B->invm, p, B->v);
    v_cross(rb, p, c); m_vec(IB, c, dw); v_sub(B->w, dw, B->w);
}

static void rel_vel(const body_t *A, const body_t *B, const double ra[3], const double rb[3], double vr[3]) {
    double wa[3], wb[3];
    v_cross(A->w, ra, wa); v_cross(B->w, rb, wb);
    for (int i = 0; i < 3; ++i) vr[i] = (A->v[i] + wa[i]) - (B->v[i] + wb[i]);
}

static void sweep(body_t *bodies, row_t *rows, int nr, double (*Iinv)[9], int use_bias) {
    for (int r = 0; r < nr; ++r) {
        row_t *R = &rows[r];
        if (R->kn == 0.0) continue;
        body_t *A = &bodies[R->a], *B = &bodies[R->b];
        double vr[3], p[3];
        /* normal row: lambda_n >= 0 */
        rel_vel(A, B, R->ra, R->rb, vr);
        double vn = v_dot(R->n, vr) + (use_bias ? R->bias : 0.0);
        double ln = R->ln - R->kn * vn;
        if (ln < 0.0) ln = 0.0;
        double dl = ln - R->ln;
        R->ln = ln;
        v_scale(R->n, dl, p);
        apply_impulse(A, B, Iinv[R->a], Iinv[R->b], R->ra, R->rb, p);
        /* friction rows, projected jointly on the disk |lambda_t| <= mu lambda_n */
        rel_vel(A, B, R->ra, R->rb, vr);
        double l1 = R->lt1 - R->kt1 * v_dot(R->t1, vr);
        double l2 = R->lt2 - R->kt2 * v_dot(R->t2, vr);
        double lim = R->mu * R->ln;
        double lt = sqrt(l1 * l1 + l2 * l2);
        if (lt > lim) {
            double s = lt > 0.0 ? lim / lt : 0.0;
            l1 *= s; l2 *= s;
        }
        double d1 = l1 - R->lt1, d2 = l2 - R->lt2;
        R->lt1 = l1; R->lt2 = l2;
        for (int i = 0; i < 3; ++i) p[i] = d1 * R->t1[i] + d2 * R->t2[i];
        apply_impulse(A, B, Iinv[R->a], Iinv[R->b], R->ra, R->rb, p);
    }
}

/* R18: one Jacobi sweep over the env's rows */
static void sweep_jacobi(body_t *bodies, row_t *rows, int nr, double (*Iinv)[9], int use_bias) {
    int na = 0;
    for (int r = 0; r < nr; ++r) na += rows[r].kn != 0.0;
    if (na == 0) return;
    const double om = 1.0 / (double)na;
    double *d = (double *)malloc(sizeof(double) * 3 * nr);
    for (int r = 0; r < nr; ++r) {   /* block updates at the sweep's start velocities */
        const row_t *R = &rows[r];
        d[3 * r] = d[3 * r + 1] = d[3 * r + 2] = 0.0;
        if (R->kn == 0.0) continue;
        body_t A = bodies[R->a], B = bodies[R->b];   /* copies: the sweep-start state */
        double vr[3], p[3];
        rel_vel(&A, &B, R->ra, R->rb, vr);
        double vn = v_dot(R->n, vr) + (use_bias ? R->bias : 0.0);
        double ln = R->ln - R->kn * vn;
        if (ln < 0.0) ln = 0.0;
        const double dl = ln - R->ln;
        v_scale(R->n, dl, p);
        apply_impulse(&A, &B, Iinv[R->a], Iinv[R->b], R->ra, R->rb, p);
        rel_vel(&A, &B, R->ra, R->rb, vr);
        double l1 = R->lt1 - R->kt1 * v_dot(R->t1, vr);
        double l2 = R->lt2 - R->kt2 * v_dot(R->t2, vr);
        const double lim = R->mu * ln;
        const double lt = sqrt(l1 * l1 + l2 * l2);
        if (lt > lim) {
            const double s = lt > 0.0 ? lim / lt : 0.0;
            l1 *= s; l2 *= s;
        }
        d[3 * r] = dl; d[3 * r + 1] = l1 - R->lt1; d[3 * r + 2] = l2 - R->lt2;
    }
    for (int r = 0; r < nr; ++r) {   /* all of them, weighted */
        row_t *R = &rows[r];
        if (R->kn == 0.0) continue;
        const double dl = om * d[3 * r], d1 = om * d[3 * r + 1], d2 = om * d[3 * r + 2];
        R->ln += dl; R->lt1 += d1; R->lt2 += d2;
        double p[3];
        for (int i = 0; i < 3; ++i) p[i] = dl * R->n[i] + d1 * R->t1[i] + d2 * R->t2[i];
        apply_impulse(&bodies[R->a], &bodies[R->b], Iinv[R->a], Iinv[R->b], R->ra, R->rb, p);
    }
    free(d);
}

static void env_substep(or_world *w, int e, double hs, int n_iters) {
    const env_t *E = &w->envs[e];
    body_t *bodies = &w->bodies[E->first_body];
    int nb = E->n_bodies;
    double (*Iw)[9] = malloc(sizeof(double) * 9 * nb);
    double (*Iinv)[9] = malloc(sizeof(double) * 9 * nb);
    double (*com)[3] = malloc(sizeof(double) * 3 * nb);
    /* 1. external forces (gravity, applied force and torque, gyroscopic term) */
    for (int i = 0; i < nb; ++i) {
        body_t *b = &bodies[i];
        body_world_inertia(b, Iw[i], Iinv[i]);
        body_com_world(b, com[i]);
        if (b->type == 2) {
            for (int k = 0; k < 3; ++k) b->v[k] += hs * (w->cfg.gravity[k] + b->force[k] / b->mass);
            double Lw[3], gyro[3], t[3], dw[3];
            m_vec(Iw[i], b->w, Lw);
            v_cross(b->w, Lw, gyro);
            v_sub(b->torque, gyro, t);
            m_vec(Iinv[i], t, dw);
            v_axpy(hs, dw, b->w);
        } else if (b->type == 3) {
            double Ia[3];
            m_vec(Iw[i], b->axis, Ia);
            double Iaa = v_dot(b->axis, Ia);
            v_axpy(hs * v_dot(b->axis, b->torque) / Iaa, b->axis, b->w);
        }
    }
    /* 3. prep: rows from the contacts of every pair of the env, in pair order -- in a pile
       env, in colour order (R20): the pairs with contacts are coloured greedily in pair
       order, each taking the lowest colour no earlier pair sharing one of its movable bodies
       took (64 colours at most; the last one gathers every pair left over), and their rows
       follow colour by colour, in pair order within a colour.  Pairs of one colour share no
       movable body, so solving them in any order, or at once, gives these same updates. */
    const int np_e = env_np(w, e);
    pair_t *pairs_e = env_pairs(w, e);
    const pair_contacts_t *pcs_e = env_pcs(w, e);
    int *order = (int *)malloc(sizeof(int) * (np_e > 0 ? np_e : 1));
    int n_order = 0;
    if (E->pile) {
        unsigned long long *used = (unsigned long long *)calloc(nb > 0 ? nb : 1, sizeof(unsigned long long));
        int n_colors = 0;
        for (int p = 0; p < np_e; ++p) {
            pairs_e[p].color = -1;
            if (pcs_e[p].n == 0) continue;
            const int la = pairs_e[p].a - E->first_body, lb = pairs_e[p].b - E->first_body;
            const int ma = movable(&bodies[la]), mb = movable(&bodies[lb]);
            const unsigned long long taken = (ma ? used[la] : 0ull) | (mb ? used[lb] : 0ull);
            int c = 0;
            while (c < 63 && ((taken >> c) & 1ull)) ++c;
            pairs_e[p].color = c;
            if (ma) used[la] |= 1ull << c;
            if (mb) used[lb] |= 1ull << c;
            if (c + 1 > n_colors) n_colors = c + 1;
        }
        for (int c = 0; c < n_colors; ++c)
            for (int p = 0; p < np_e; ++p)
                if (pairs_e[p].color == c) order[n_order++] = p;
        free(used);
    } else {
        for (int p = 0; p < np_e; ++p) order[n_order++] = p;
    }
    int nr = 0;
    for (int p = 0; p < np_e; ++p) nr += pcs_e[p].n;
    row_t *rows = (row_t *)calloc(nr > 0 ? nr : 1, sizeof(row_t));
    int r = 0;
    for (int q = 0; q < n_order; ++q) {
        const int p = order[q];
        const pair_t *P = &pairs_e[p];
        const pair_contacts_t *pc = &pcs_e[p];
        int la = P->a - E->first_body, lb = P->b - E->first_body;
        for (int i = 0; i < pc->n; ++i, ++r) {
            const or_contact *c = &pc->c[i];
            row_t *R = &rows[r];
            R->a = la; R->b = lb;
            v_sub(c->xa, com[la], R->ra);
            v_sub(c->xb, com[lb], R->rb);
            memcpy(R->n, c->n, sizeof R->n);
            margin_t tm = {INFINITY, INFINITY};
            tangent_basis(R->n, R->t1, R->t2, &tm);
            if (tm.dot < w->env_mdot[e]) w->env_mdot[e] = tm.dot;
            R->kn = eff_mass(&bodies[la], &bodies[lb], Iinv[la], Iinv[lb], R->ra, R->rb, R->n);
            R->kt1 = eff_mass(&bodies[la], &bodies[lb], Iinv[la], Iinv[lb], R->ra, R->rb, R->t1);
            R->kt2 = eff_mass(&bodies[la], &bodies[lb], Iinv[la], Iinv[lb], R->ra, R->rb, R->t2);
            R->bias = (c->phi > 0.0) ? c->phi / hs : w->cfg.baumgarte * c->phi / hs;
            R->mu = P->mu;
        }
    }
    /* 4. Gauss-Seidel sweeps (R9), or Jacobi sweeps (R18) */
    for (int it = 0; it < n_iters; ++it) {
        if (w->cfg.solver == 1) sweep_jacobi(bodies, rows, nr, Iinv, 1);
        else sweep(bodies, rows, nr, Iinv, 1);
    }
    /* 5. integrate */
    for (int i = 0; i < nb; ++i) {
        body_t *b = &bodies[i];
        if (b->type == 0) continue;
        if ((b->type == 2 || b->type == 3) && w->cfg.max_angvel > 0.0) {
            double wn = v_norm(b->w);
            if (wn > w->cfg.max_angvel) v_scale(b->w, w->cfg.max_angvel / wn, b->w);
        }
        double c[3], R[9], rc[3];
        memcpy(c, com[i], sizeof c);
        v_axpy(hs, b->v, c);
        double wq[4] = {b->w[0], b->w[1], b->w[2], 0.0}, dq[4];
        /* (omega, 0) (x) q */
        dq[0] = wq[3] * b->q[0] + b->q[3] * wq[0] + wq[1] * b->q[2] - wq[2] * b->q[1];
        dq[1] = wq[3] * b->q[1] + b->q[3] * wq[1] + wq[2] * b->q[0] - wq[0] * b->q[2];
        dq[2] = wq[3] * b->q[2] + b->q[3] * wq[2] + wq[0] * b->q[1] - wq[1] * b->q[0];
        dq[3] = wq[3] * b->q[3] - (wq[0] * b->q[0] + wq[1] * b->q[1] + wq[2] * b->q[2]);
        for (int k = 0; k < 4; ++k) b->q[k] += 0.5 * hs * dq[k];
        q_normalize(b->q);
        q_to_m(b->q, R);
        m_vec(R, b->com_b, rc);
        v_sub(c, rc, b->p);
    }
    /* 6. optional bias-free sweeps */
    for (int it = 0; it < w->cfg.n_vel_iters; ++it) {
        if (w->cfg.solver == 1) sweep_jacobi(bodies, rows, nr, Iinv, 0);
        else sweep(bodies, rows, nr, Iinv, 0);
    }
    /* friction-cone record of this solve: (lambda_n, |lambda_t|, mu) per row */
    double *rec = (double *)malloc(sizeof(double) * 3 * (nr > 0 ? nr : 1));
    for (int k = 0; k < nr; ++k) {
        rec[3 * k] = rows[k].ln;
        rec[3 * k + 1] = sqrt(rows[k].lt1 * rows[k].lt1 + rows[k].lt2 * rows[k].lt2);
        rec[3 * k + 2] = rows[k].mu;
    }
    free(w->imp[e]);
    w->imp[e] = rec;
    w->imp_n[e] = nr;
    free(rows); free(Iw); free(Iinv); free(com); free(order);
}

int or_substep(or_world *w, double hs, int n_iters, int detect) {
    if (detect) or_collide(w);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(team_size(w->cfg.n_threads))
#endif
    for (int e = 0; e < w->n_envs; ++e) env_substep(w, e, hs, n_iters);
    return 0;
}

int or_step(or_world *w, int n_substeps, int n_iters) {
    double hs = w->cfg.dt / (double)n_substeps;
    for (int s = 0; s < n_substeps; ++s) or_substep(w, hs, n_iters, 1);
    return 0;
}

int or_get_state(const or_world *w, double *pos, double *quat, double *linvel, double *angvel) {
    for (int i = 0; i < w->n_bodies; ++i) {
        const body_t *b = &w->bodies[i];
        memcpy(pos + 3 * i, b->p, 3 * sizeof(double));
        memcpy(quat + 4 * i, b->q, 4 * sizeof(double));
        memcpy(linvel + 3 * i, b->v, 3 * sizeof(double));
        memcpy(angvel + 3 * i, b->w, 3 * sizeof(double));
    }
    return 0;
}

int or_set_state(or_world *w, const double *pos, const double *quat, const double *linvel,
                 const double *angvel) {
    for (int i = 0; i < w->n_bodies; ++i) {
        body_t *b = &w->bodies[i];
        memcpy(b->p, pos + 3 * i, 3 * sizeof(double));
        memcpy(b->q, quat + 4 * i, 4 * sizeof(double));
        q_normalize(b->q);
        memcpy(b->v, linvel + 3 * i, 3 * sizeof(double));
        memcpy(b->w, angvel + 3 * i, 3 * sizeof(double));
    }
    return 0;
}

int or_get_impulses(const or_world *w, int env, double *out, int cap, int *n_out) {
    int n = w->imp_n[env];
    for (int k = 0; k < n && k < cap; ++k) memcpy(out + 3 * k, w->imp[env] + 3 * k, 3 * sizeof(double));
    *n_out = n;
    return n > cap ? -1 : 0;
}

/* ==================================================================================== */
/* Differentiable rollout: reverse mode of substeps whose discrete decisions are held    */
/* fixed by a tape.                                                                       */
/* ==================================================================================== */
/*
 * Scope: an env is differentiable when exactly one of its bodies is dynamic and that body
 * is the point-sampled body a of every pair of the env; its partners are static or
 * kinematic (prescribed motion, no adjoint); n_vel_iters = 0.  Envs without a dynamic
 * body are allowed and carry no adjoint.
 *
 * The tape of a rollout of S substeps over E envs with K sweeps each:
 *   c_off[s*E + e] .. c_off[s*E + e + 1]: the contacts of env e in substep s, in solve
 *     order, each 6 ints: sample, pair (global id), SDF cell i, j, k, flags (bit 0: t1
 *     from n x e_x, bit 1: phi > 0, the speculative bias);
 *   r_bits[K*c + it] for contact c (index into the records) and sweep it: bit 0 the
 *     normal impulse is positive after the row, bit 1 the friction impulse was projected
 *     onto the disk |lambda_t| <= mu lambda_n;
 *   b_bits[s*E + e]: bit 0 the dynamic body's |omega| was clamped at integration.
 * Recording takes each decision as the oracle's forward does (its own detection and
 * Algorithm 1 each substep).  Replaying evaluates the same formulas with the taped
 * decisions -- the trilinear polynomial of the taped cell is used even a little outside
 * that cell -- so a replay is a smooth function of the initial state, of the dynamic
 * bodies' masses (inertia scaled with mass at fixed geometry) and of the pairs' friction
 * coefficients, equal to the plain forward at the recorded point.  The adjoint below is
 * the exact reverse mode of a replay.
 */
struct diff_tape {
    int S, E, K;
    double hs;
    int *c_off;
    int *c_rec;
    int n_c, cap_c;
    unsigned char *r_bits;
    unsigned char *b_bits;
};

static void diff_tape_free(or_world *w) {
    if (!w->tape) return;
    free(w->tape->c_off); free(w->tape->c_rec); free(w->tape->r_bits); free(w->tape->b_bits);
    free(w->tape);
    w->tape = NULL;
}

static struct diff_tape *diff_tape_new(int S, int E, int K, double hs) {
    struct diff_tape *T = (struct diff_tape *)calloc(1, sizeof(struct diff_tape));
    T->S = S; T->E = E; T->K = K; T->hs = hs;
    T->c_off = (int *)calloc((size_t)S * E + 1, sizeof(int));
    T->b_bits = (unsigned char *)calloc((size_t)S * E + 1, 1);
    return T;
}

/* the dynamic body of env e (global id); -2 none; -1 the env is not differentiable */
static int diff_env_body(const or_world *w, int e) {
    const env_t *E = &w->envs[e];
    int dyn = -2;
    for (int i = 0; i < E->n_bodies; ++i) {
        const int t = w->bodies[E->first_body + i].type;
        if (t == 3) return -1;
        if (t == 2) {
            if (dyn >= 0) return -1;
            dyn = E->first_body + i;
        }
    }
    if (dyn >= 0 && E->pile) return -1;   /* piles are not differentiable */
    if (dyn >= 0)
        for (int p = 0; p < E->n_pairs; ++p)
            if (w->pairs[E->first_pair + p].a != dyn) return -1;
    return dyn;
}

/* the 8 nodes of a cell, baked now if the grid is lazy */
static void diff_cell_nodes(or_world *w, asset_t *ab, const int c[3], double v[2][2][2]) {
    grid_t *g = &ab->grid;
    for (int k = 0; k < 8; ++k) {
        const long long id = gidx(g, c[0] + (k & 1), c[1] + ((k >> 1) & 1), c[2] + ((k >> 2) & 1));
        if (g->lazy && g->done[id] != 1) {
            float lo[3] = {(float)g->lo[0], (float)g->lo[1], (float)g->lo[2]};
            double val;
            or_bake_nodes(ab->V, ab->T, ab->nt, lo, (float)g->h, g->dims, &id, 1, &val, 1);
            g->val[id] = val;
            g->done[id] = 1;
        }
        v[(k >> 2) & 1][(k >> 1) & 1][k & 1] = g->val[id];
    }
    (void)w;
}

/* value, gradient and Hessian of the trilinear polynomial of cell c at x (grid frame);
 * f may fall slightly outside [0, 1] on a replay.  Within a cell the Hessian has a zero
 * diagonal; its mixed terms are the bilinear blends of the cell's second differences. */
static void diff_trilinear(or_world *w, asset_t *ab, const int c[3], const double x[3], double *phi,
                           double grad[3], double H[9]) {
    const grid_t *g = &ab->grid;
    double f[3], v[2][2][2];
    for (int a = 0; a < 3; ++a) f[a] = (x[a] - g->lo[a]) / g->h - (double)c[a];
    diff_cell_nodes(w, ab, c, v);
    const double wx[2] = {1 - f[0], f[0]}, wy[2] = {1 - f[1], f[1]}, wz[2] = {1 - f[2], f[2]};
    double p = 0, gx = 0, gy = 0, gz = 0, hxy = 0, hxz = 0, hyz = 0;
    for (int dk = 0; dk < 2; ++dk)
        for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) p += wx[di] * wy[dj] * wz[dk] * v[dk][dj][di];
    for (int dk = 0; dk < 2; ++dk)
        for (int dj = 0; dj < 2; ++dj) gx += wy[dj] * wz[dk] * (v[dk][dj][1] - v[dk][dj][0]);
    for (int dk = 0; dk < 2; ++dk)
        for (int di = 0; di < 2; ++di) gy += wx[di] * wz[dk] * (v[dk][1][di] - v[dk][0][di]);
    for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di) gz += wx[di] * wy[dj] * (v[1][dj][di] - v[0][dj][di]);
    for (int dk = 0; dk < 2; ++dk) hxy += wz[dk] * (v[dk][1][1] - v[dk][1][0] - v[dk][0][1] + v[dk][0][0]);
    for (int dj = 0; dj < 2; ++dj) hxz += wy[dj] * (v[1][dj][1] - v[1][dj][0] - v[0][dj][1] + v[0][dj][0]);
    for (int di = 0; di < 2; ++di) hyz += wx[di] * (v[1][1][di] - v[1][0][di] - v[0][1][di] + v[0][0][di]);
    *phi = p;
    grad[0] = gx / g->h; grad[1] = gy / g->h; grad[2] = gz / g->h;
    const double ih2 = 1.0 / (g->h * g->h);
    H[0] = 0; H[1] = hxy * ih2; H[2] = hxz * ih2;
    H[3] = hxy * ih2; H[4] = 0; H[5] = hyz * ih2;
    H[6] = hxz * ih2; H[7] = hyz * ih2; H[8] = 0;
}

/* one contact row of the dynamic body (all quantities world frame) */
typedef struct {
    int pair, flags, cell[3], live;
    double s[3];                       /* sample, body-a frame */
    double xbl[3], phi, g[3], H[9], gn, nb[3];
    double xa[3], xbw[3], n[3];
    double ra[3], rb[3], uo[3], tr[3], tn;
    double d[3][3], a[3][3], b[3][3], k[3];   /* directions n, t1, t2; r x d; I^-1 (r x d); 1/den */
    double bias, e[3], mu;
} drow_t;

/* forward intermediates of one env substep */
typedef struct {
    int ia;                          /* dynamic body (global id) or < 0 */
    double q0[4], R[9], com[3], Iw[9], Ii[9];
    double v0[3], w0[3], v1[3], w1[3], Lw[3], tq[3];
    drow_t *rows;
    int nr, c0;                      /* rows and the index of the first tape record */
    double *upd;                     /* per (sweep, row): v, w, lambda before the update (9) */
    double vf[3], wf[3], wc[3];
    double cp[3], qt[4], q1[4], R1[9];
    int clamped;
} dfwd_t;

static void m_sandwich(const double R[9], const double S[9], double M[9]) {   /* R S R^T */
    double Rt[9], t[9];
    m_transpose(R, Rt);
    m_mul(R, S, t);
    m_mul(t, Rt, M);
}

/* geometry and row of one taped contact at the current state */
static void diff_build_row(or_world *w, const body_t *A, const dfwd_t *F, drow_t *D, double hs) {
    const pair_t *P = &w->pairs[D->pair];
    const body_t *B = &w->bodies[P->b];
    asset_t *ab = &w->assets[B->asset];
    double RB[9], RBt[9], d[3], H[9];
    q_to_m(B->q, RB);
    m_transpose(RB, RBt);
    m_vec(F->R, D->s, D->xa);
    v_add(D->xa, A->p, D->xa);
    v_sub(D->xa, B->p, d);
    m_vec(RBt, d, D->xbl);
    diff_trilinear(w, ab, D->cell, D->xbl, &D->phi, D->g, H);
    memcpy(D->H, H, sizeof H);
    D->gn = v_norm(D->g);
    v_scale(D->g, 1.0 / D->gn, D->nb);
    m_vec(RB, D->nb, D->n);
    for (int i = 0; i < 3; ++i) D->xbw[i] = D->xa[i] - D->phi * D->n[i];
    v_sub(D->xa, F->com, D->ra);
    double comB[3], wr[3];
    body_com_world(B, comB);
    v_sub(D->xbw, comB, D->rb);
    v_cross(B->w, D->rb, wr);
    v_add(B->v, wr, D->uo);
    /* tangent basis (R11) with the taped branch */
    if (D->flags & 1) { D->tr[0] = 0; D->tr[1] = D->n[2]; D->tr[2] = -D->n[1]; }
    else { D->tr[0] = -D->n[2]; D->tr[1] = 0; D->tr[2] = D->n[0]; }
    D->tn = v_norm(D->tr);
    memcpy(D->d[0], D->n, sizeof D->n);
    v_scale(D->tr, 1.0 / D->tn, D->d[1]);
    v_cross(D->n, D->d[1], D->d[2]);
    D->live = 1;
    for (int j = 0; j < 3; ++j) {
        v_cross(D->ra, D->d[j], D->a[j]);
        m_vec(F->Ii, D->a[j], D->b[j]);
        const double den = A->invm + v_dot(D->a[j], D->b[j]);
        D->k[j] = den > 0.0 ? 1.0 / den : 0.0;
        D->e[j] = -v_dot(D->d[j], D->uo);
    }
    if (D->k[0] == 0.0) D->live = 0;
    D->bias = (D->flags & 2) ? D->phi / hs : w->cfg.baumgarte * D->phi / hs;
    D->mu = P->mu;
}

/* one row update of the sweep (R9) with the given decisions (record: bits computed) */
static void diff_row_fwd(const drow_t *D, double invm, double v[3], double wv[3], double lam[3],
                         unsigned char *bits, int replay) {
    const double jv = v_dot(D->d[0], v) + v_dot(D->a[0], wv) + D->bias + D->e[0];
    const double u = lam[0] - D->k[0] * jv;
    int act;
    if (replay) act = (*bits & 1) != 0; else act = u > 0.0;
    const double ln = act ? u : 0.0;
    const double dl = ln - lam[0];
    double vm[3], wm[3];
    for (int i = 0; i < 3; ++i) { vm[i] = v[i] + invm * dl * D->d[0][i]; wm[i] = wv[i] + dl * D->b[0][i]; }
    const double j1 = v_dot(D->d[1], vm) + v_dot(D->a[1], wm) + D->e[1];
    const double j2 = v_dot(D->d[2], vm) + v_dot(D->a[2], wm) + D->e[2];
    const double t1 = lam[1] - D->k[1] * j1, t2 = lam[2] - D->k[2] * j2;
    const double lim = D->mu * ln, tn = sqrt(t1 * t1 + t2 * t2);
    int proj;
    if (replay) proj = (*bits & 2) != 0; else proj = tn > lim;
    const double s = proj ? lim / tn : 1.0;
    const double l1 = s * t1, l2 = s * t2;
    const double e1 = l1 - lam[1], e2 = l2 - lam[2];
    for (int i = 0; i < 3; ++i) {
        v[i] = vm[i] + invm * (e1 * D->d[1][i] + e2 * D->d[2][i]);
        wv[i] = wm[i] + e1 * D->b[1][i] + e2 * D->b[2][i];
    }
    lam[0] = ln; lam[1] = l1; lam[2] = l2;
    if (!replay) *bits = (unsigned char)((act ? 1 : 0) | (proj ? 2 : 0));
}

/* (omega, 0) (x) q */
static void omega_q(const double wv[3], const double q[4], double dq[4]) {
    dq[0] = q[3] * wv[0] + wv[1] * q[2] - wv[2] * q[1];
    dq[1] = q[3] * wv[1] + wv[2] * q[0] - wv[0] * q[2];
    dq[2] = q[3] * wv[2] + wv[0] * q[1] - wv[1] * q[0];
    dq[3] = -(wv[0] * q[0] + wv[1] * q[1] + wv[2] * q[2]);
}

/* Forward of env e in substep si with tape T: record (contacts from the world's current
 * detection, decisions computed) or replay (contacts and decisions from the tape).  The
 * bodies' states advance.  F (optional) keeps what the adjoint needs. */
static int diff_env_forward(or_world *w, int e, int si, int replay, dfwd_t *F, int keep_updates) {
    struct diff_tape *T = w->tape;
    const env_t *E = &w->envs[e];
    const double hs = T->hs;
    const int K = T->K;
    memset(F, 0, sizeof *F);
    F->ia = diff_env_body(w, e);
    if (F->ia == -1) return -1;
    const int slot = si * T->E + e;
    if (F->ia >= 0) {
        body_t *A = &w->bodies[F->ia];
        /* 1. external forces at the substep's start */
        memcpy(F->q0, A->q, sizeof F->q0);
        q_to_m(A->q, F->R);
        body_com_world(A, F->com);
        m_sandwich(F->R, A->Ib, F->Iw);
        m_sandwich(F->R, A->Ib_inv, F->Ii);
        memcpy(F->v0, A->v, sizeof F->v0);
        memcpy(F->w0, A->w, sizeof F->w0);
        for (int k = 0; k < 3; ++k) F->v1[k] = A->v[k] + hs * (w->cfg.gravity[k] + A->force[k] / A->mass);
        double gy[3], dw[3];
        m_vec(F->Iw, A->w, F->Lw);
        v_cross(A->w, F->Lw, gy);
        v_sub(A->torque, gy, F->tq);
        m_vec(F->Ii, F->tq, dw);
        for (int k = 0; k < 3; ++k) F->w1[k] = A->w[k] + hs * dw[k];
        /* 2. contacts (taped or recorded now) and their rows */
        if (!replay) {
            int n = 0;
            for (int p = 0; p < E->n_pairs; ++p) n += w->pc[E->first_pair + p].n;
            if (T->n_c + n > T->cap_c) {
                T->cap_c = 2 * (T->n_c + n) + 64;
                T->c_rec = (int *)realloc(T->c_rec, sizeof(int) * 6 * T->cap_c);
                T->r_bits = (unsigned char *)realloc(T->r_bits, (size_t)K * T->cap_c);
            }
            T->c_off[slot] = T->n_c;
            for (int p = 0; p < E->n_pairs; ++p) {
                const int pi = E->first_pair + p;
                const pair_contacts_t *pc = &w->pc[pi];
                const body_t *B = &w->bodies[w->pairs[pi].b];
                const grid_t *g = &w->assets[B->asset].grid;
                for (int i = 0; i < pc->n; ++i) {
                    int *rec = T->c_rec + 6 * T->n_c;
                    rec[0] = pc->c[i].sample;
                    rec[1] = pi;
                    double RB[9], RBt[9], xw[3], d[3], xb[3], s3[3];
                    load3(w->assets[A->asset].S + 3 * rec[0], s3);
                    q_to_m(B->q, RB); m_transpose(RB, RBt);
                    m_vec(F->R, s3, xw); v_add(xw, A->p, xw);
                    v_sub(xw, B->p, d); m_vec(RBt, d, xb);
                    for (int a = 0; a < 3; ++a) {
                        int ci = (int)floor((xb[a] - g->lo[a]) / g->h);
                        if (ci > g->dims[a] - 2) ci = g->dims[a] - 2;
                        if (ci < 0) ci = 0;
                        rec[2 + a] = ci;
                    }
                    rec[5] = (fabs(pc->c[i].n[0]) < 0.57735 ? 1 : 0) | (pc->c[i].phi > 0.0 ? 2 : 0);
                    T->n_c++;
                }
            }
            T->c_off[slot + 1] = T->n_c;
        }
        F->c0 = T->c_off[slot];
        F->nr = T->c_off[slot + 1] - F->c0;
        F->rows = (drow_t *)calloc(F->nr > 0 ? F->nr : 1, sizeof(drow_t));
        for (int r = 0; r < F->nr; ++r) {
            const int *rec = T->c_rec + 6 * (F->c0 + r);
            drow_t *D = &F->rows[r];
            D->pair = rec[1];
            D->cell[0] = rec[2]; D->cell[1] = rec[3]; D->cell[2] = rec[4];
            D->flags = rec[5];
            load3(w->assets[A->asset].S + 3 * rec[0], D->s);
            diff_build_row(w, A, F, D, hs);
        }
        /* 3. sweeps */
        double *lam = (double *)calloc(3 * (F->nr > 0 ? F->nr : 1), sizeof(double));
        double v[3], wv[3];
        memcpy(v, F->v1, sizeof v);
        memcpy(wv, F->w1, sizeof wv);
        if (keep_updates) F->upd = (double *)malloc(sizeof(double) * 9 * (size_t)K * (F->nr > 0 ? F->nr : 1));
        for (int it = 0; it < K; ++it)
            for (int r = 0; r < F->nr; ++r) {
                if (keep_updates) {
                    double *u = F->upd + 9 * ((size_t)it * F->nr + r);
                    memcpy(u, v, 3 * sizeof(double)); memcpy(u + 3, wv, 3 * sizeof(double));
                    memcpy(u + 6, lam + 3 * r, 3 * sizeof(double));
                }
                if (!F->rows[r].live) continue;
                diff_row_fwd(&F->rows[r], A->invm, v, wv, lam + 3 * r, T->r_bits + (size_t)K * (F->c0 + r) + it, replay);
            }
        free(lam);
        memcpy(F->vf, v, sizeof v);
        memcpy(F->wf, wv, sizeof wv);
        /* 4. integration (R10) */
        memcpy(F->wc, wv, sizeof wv);
        const double wn = v_norm(wv);
        if (!replay) T->b_bits[slot] = (w->cfg.max_angvel > 0.0 && wn > w->cfg.max_angvel) ? 1 : 0;
        F->clamped = T->b_bits[slot] & 1;
        if (F->clamped) v_scale(wv, w->cfg.max_angvel / wn, F->wc);
        for (int k = 0; k < 3; ++k) F->cp[k] = F->com[k] + hs * F->vf[k];
        double dq[4];
        omega_q(F->wc, A->q, dq);
        for (int k = 0; k < 4; ++k) F->qt[k] = A->q[k] + 0.5 * hs * dq[k];
        memcpy(F->q1, F->qt, sizeof F->qt);
        q_normalize(F->q1);
        q_to_m(F->q1, F->R1);
        double rc[3];
        m_vec(F->R1, A->com_b, rc);
        v_sub(F->cp, rc, A->p);
        memcpy(A->q, F->q1, sizeof F->q1);
        memcpy(A->v, F->vf, sizeof F->vf);
        memcpy(A->w, F->wc, sizeof F->wc);
    }
    /* kinematic partners follow their prescribed velocity (R10) */
    for (int i = 0; i < E->n_bodies; ++i) {
        body_t *b = &w->bodies[E->first_body + i];
        if (b->type != 1) continue;
        double c[3], R[9], rc[3], dq[4];
        body_com_world(b, c);
        v_axpy(hs, b->v, c);
        omega_q(b->w, b->q, dq);
        for (int k = 0; k < 4; ++k) b->q[k] += 0.5 * hs * dq[k];
        q_normalize(b->q);
        q_to_m(b->q, R);
        m_vec(R, b->com_b, rc);
        v_sub(c, rc, b->p);
    }
    return 0;
}

static void dfwd_free(dfwd_t *F) { free(F->rows); free(F->upd); F->rows = NULL; F->upd = NULL; }

/* adjoint of R = q_to_m(q) for the polynomial of q_to_m: qb += sum Rb_ij dR_ij/dq */
static void q_to_m_vjp(const double q[4], const double Rb[9], double qb[4]) {
    const double x = q[0], y = q[1], z = q[2], w = q[3];
    qb[0] += 2 * y * Rb[1] + 2 * z * Rb[2] + 2 * y * Rb[3] - 4 * x * Rb[4] - 2 * w * Rb[5] + 2 * z * Rb[6] +
             2 * w * Rb[7] - 4 * x * Rb[8];
    qb[1] += -4 * y * Rb[0] + 2 * x * Rb[1] + 2 * w * Rb[2] + 2 * x * Rb[3] + 2 * z * Rb[5] - 2 * w * Rb[6] +
             2 * z * Rb[7] - 4 * y * Rb[8];
    qb[2] += -4 * z * Rb[0] - 2 * w * Rb[1] + 2 * x * Rb[2] + 2 * w * Rb[3] - 4 * z * Rb[4] + 2 * y * Rb[5] +
             2 * x * Rb[6] + 2 * y * Rb[7];
    qb[3] += -2 * z * Rb[1] + 2 * y * Rb[2] + 2 * z * Rb[3] - 2 * x * Rb[5] - 2 * y * Rb[6] + 2 * x * Rb[7];
}

/* y = M x:  xb += M^T yb,  Mb += yb x^T */
static void mv_vjp(const double M[9], const double x[3], const double yb[3], double xb[3], double Mb[9]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            if (xb) xb[j] += M[3 * i + j] * yb[i];
            if (Mb) Mb[3 * i + j] += yb[i] * x[j];
        }
}

/* r = a x b:  ab += b x rb,  bb += rb x a */
static void cross_vjp(const double a[3], const double b[3], const double rb[3], double ab[3], double bb[3]) {
    double t[3];
    if (ab) { v_cross(b, rb, t); v_add(ab, t, ab); }
    if (bb) { v_cross(rb, a, t); v_add(bb, t, bb); }
}

/* M = R S R^T (S symmetric):  Rb += (Mb + Mb^T) R S,  Sb += R^T Mb R */
static void sandwich_vjp(const double R[9], const double S[9], const double Mb[9], double Rb[9], double Sb[9]) {
    double Ms[9], t[9], Rt[9], u[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Ms[3 * i + j] = Mb[3 * i + j] + Mb[3 * j + i];
    m_mul(Ms, R, t);
    m_mul(t, S, u);
    for (int k = 0; k < 9; ++k) Rb[k] += u[k];
    if (Sb) {
        m_transpose(R, Rt);
        m_mul(Rt, Mb, t);
        m_mul(t, R, u);
        for (int k = 0; k < 9; ++k) Sb[k] += u[k];
    }
}

/* adjoints of one row's data, accumulated over the sweeps */
typedef struct {
    double d[3][3], a[3][3], b[3][3], k[3], bias, e[3], mu;
} drow_bar_t;

/* reverse of diff_row_fwd: (v, w, lam) before the update in u; vb, wb, lb hold the
 * adjoints of the outputs and receive those of the inputs; row adjoints into RB */
static void diff_row_rev(const drow_t *D, double invm, const double *u, unsigned char bits, double vb[3],
                         double wb[3], double lb[3], drow_bar_t *RB, double *invm_b) {
    const double *v = u, *wv = u + 3, *lam = u + 6;
    /* recompute the forward of this update */
    const double jv = v_dot(D->d[0], v) + v_dot(D->a[0], wv) + D->bias + D->e[0];
    const double uu = lam[0] - D->k[0] * jv;
    const int act = bits & 1, proj = (bits & 2) != 0;
    const double ln = act ? uu : 0.0, dl = ln - lam[0];
    double vm[3], wm[3];
    for (int i = 0; i < 3; ++i) { vm[i] = v[i] + invm * dl * D->d[0][i]; wm[i] = wv[i] + dl * D->b[0][i]; }
    const double j1 = v_dot(D->d[1], vm) + v_dot(D->a[1], wm) + D->e[1];
    const double j2 = v_dot(D->d[2], vm) + v_dot(D->a[2], wm) + D->e[2];
    const double t1 = lam[1] - D->k[1] * j1, t2 = lam[2] - D->k[2] * j2;
    const double lim = D->mu * ln, tn = sqrt(t1 * t1 + t2 * t2);
    const double s = proj ? lim / tn : 1.0;
    const double l1 = s * t1, l2 = s * t2, e1 = l1 - lam[1], e2 = l2 - lam[2];
    /* v' = vm + invm (e1 d1 + e2 d2),  w' = wm + e1 b1 + e2 b2 */
    double vmb[3], wmb[3];
    memcpy(vmb, vb, sizeof vmb);
    memcpy(wmb, wb, sizeof wmb);
    const double e1b = invm * v_dot(D->d[1], vb) + v_dot(D->b[1], wb);
    const double e2b = invm * v_dot(D->d[2], vb) + v_dot(D->b[2], wb);
    for (int i = 0; i < 3; ++i) {
        RB->d[1][i] += invm * e1 * vb[i];
        RB->d[2][i] += invm * e2 * vb[i];
        RB->b[1][i] += e1 * wb[i];
        RB->b[2][i] += e2 * wb[i];
    }
    *invm_b += v_dot(vb, D->d[1]) * e1 + v_dot(vb, D->d[2]) * e2;
    /* e_k = l_k' - l_k */
    double l1b = lb[1] + e1b, l2b = lb[2] + e2b;
    double lam_b1 = -e1b, lam_b2 = -e2b;
    /* l_k' = s t_k */
    double t1b = s * l1b, t2b = s * l2b;
    double lnb = lb[0];
    if (proj) {
        const double sb = t1 * l1b + t2 * l2b;
        const double limb = sb / tn;
        const double tnb = -sb * lim / (tn * tn);
        t1b += tnb * t1 / tn;
        t2b += tnb * t2 / tn;
        RB->mu += ln * limb;
        lnb += D->mu * limb;
    }
    /* t_k = l_k - k_tk j_k */
    lam_b1 += t1b;
    lam_b2 += t2b;
    RB->k[1] -= j1 * t1b;
    RB->k[2] -= j2 * t2b;
    const double j1b = -D->k[1] * t1b, j2b = -D->k[2] * t2b;
    /* j_k = d_k . vm + a_k . wm + e_k */
    for (int i = 0; i < 3; ++i) {
        vmb[i] += j1b * D->d[1][i] + j2b * D->d[2][i];
        wmb[i] += j1b * D->a[1][i] + j2b * D->a[2][i];
        RB->d[1][i] += j1b * vm[i];
        RB->d[2][i] += j2b * vm[i];
        RB->a[1][i] += j1b * wm[i];
        RB->a[2][i] += j2b * wm[i];
    }
    RB->e[1] += j1b;
    RB->e[2] += j2b;
    /* vm = v + invm dl dn,  wm = w + dl bn */
    const double dlb = invm * v_dot(D->d[0], vmb) + v_dot(D->b[0], wmb);
    for (int i = 0; i < 3; ++i) {
        RB->d[0][i] += invm * dl * vmb[i];
        RB->b[0][i] += dl * wmb[i];
    }
    *invm_b += dl * v_dot(D->d[0], vmb);
    /* dl = ln - lam_n */
    lnb += dlb;
    double lam_b0 = -dlb;
    /* ln = max(0, u) with the taped branch */
    const double ub = act ? lnb : 0.0;
    /* u = lam_n - k_n jv */
    lam_b0 += ub;
    RB->k[0] -= jv * ub;
    const double jvb = -D->k[0] * ub;
    /* jv = dn . v + an . w + bias + e_n */
    for (int i = 0; i < 3; ++i) {
        vb[i] = vmb[i] + jvb * D->d[0][i];
        wb[i] = wmb[i] + jvb * D->a[0][i];
        RB->d[0][i] += jvb * v[i];
        RB->a[0][i] += jvb * wv[i];
    }
    RB->bias += jvb;
    RB->e[0] += jvb;
    lb[0] = lam_b0; lb[1] = lam_b1; lb[2] = lam_b2;
}

/* Reverse of one env substep.  xb = adjoint of the dynamic body's state after the
 * substep (p 3, q 4, v 3, w 3), replaced by the adjoint before it; mass_b and mu_b
 * (per global pair) accumulate.  F holds the forward intermediates (keep_updates). */
static void diff_env_reverse(or_world *w, const dfwd_t *F, double xb[13], double *mass_b, double *mu_b) {
    const body_t *A = &w->bodies[F->ia];
    const struct diff_tape *T = w->tape;
    const double hs = T->hs;
    const int K = T->K;
    const double m = A->mass;
    double qb1[4], wcb[3], vb[3], wb[3];
    memcpy(qb1, xb + 3, sizeof qb1);
    memcpy(vb, xb + 7, sizeof vb);         /* final velocities are the state's */
    memcpy(wcb, xb + 10, sizeof wcb);
    double pbt[3] = {0, 0, 0}, comb[3], Rb[9] = {0}, qb[4] = {0, 0, 0, 0};
    /* ---- integration: p' = c' - R(q') com_b, q' = qt/|qt|, qt = q + hs/2 (w,0)(x)q,
     * c' = com + hs vf, w' = wc */
    memcpy(comb, xb, 3 * sizeof(double));  /* dp'/dc' = I */
    double R1b[9] = {0};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) R1b[3 * i + j] -= xb[i] * A->com_b[j];
    q_to_m_vjp(F->q1, R1b, qb1);
    const double qn = sqrt(F->qt[0] * F->qt[0] + F->qt[1] * F->qt[1] + F->qt[2] * F->qt[2] + F->qt[3] * F->qt[3]);
    const double dq1 = F->q1[0] * qb1[0] + F->q1[1] * qb1[1] + F->q1[2] * qb1[2] + F->q1[3] * qb1[3];
    double tb[4];
    for (int k = 0; k < 4; ++k) tb[k] = (qb1[k] - F->q1[k] * dq1) / qn;
    const double hh = 0.5 * hs;
    const double *q = F->q0, *wc = F->wc;
    for (int k = 0; k < 4; ++k) qb[k] += tb[k];
    qb[0] += hh * (wc[2] * tb[1] - wc[1] * tb[2] - wc[0] * tb[3]);
    qb[1] += hh * (-wc[2] * tb[0] + wc[0] * tb[2] - wc[1] * tb[3]);
    qb[2] += hh * (wc[1] * tb[0] - wc[0] * tb[1] - wc[2] * tb[3]);
    qb[3] += hh * (wc[0] * tb[0] + wc[1] * tb[1] + wc[2] * tb[2]);
    wcb[0] += hh * (q[3] * tb[0] - q[2] * tb[1] + q[1] * tb[2] - q[0] * tb[3]);
    wcb[1] += hh * (q[2] * tb[0] + q[3] * tb[1] - q[0] * tb[2] - q[1] * tb[3]);
    wcb[2] += hh * (-q[1] * tb[0] + q[0] * tb[1] + q[3] * tb[2] - q[2] * tb[3]);
    for (int i = 0; i < 3; ++i) vb[i] += hs * xb[i];     /* c' = com + hs vf */
    if (F->clamped) {                                    /* wc = wf max / |wf| */
        const double wn = v_norm(F->wf), s = w->cfg.max_angvel / wn;
        double u[3], d;
        v_scale(F->wf, 1.0 / wn, u);
        d = v_dot(u, wcb);
        for (int i = 0; i < 3; ++i) wb[i] = s * (wcb[i] - u[i] * d);
    } else {
        memcpy(wb, wcb, sizeof wb);
    }
    /* ---- sweeps, last update first; the final impulses carry no adjoint */
    const int nr = F->nr;
    double *lb = (double *)calloc(3 * (nr > 0 ? nr : 1), sizeof(double));
    drow_bar_t *RBr = (drow_bar_t *)calloc(nr > 0 ? nr : 1, sizeof(drow_bar_t));
    double invm_b = 0.0;
    for (int it = K - 1; it >= 0; --it)
        for (int r = nr - 1; r >= 0; --r) {
            if (!F->rows[r].live) continue;
            diff_row_rev(&F->rows[r], A->invm, F->upd + 9 * ((size_t)it * nr + r),
                         T->r_bits[(size_t)K * (F->c0 + r) + it], vb, wb, lb + 3 * r, &RBr[r], &invm_b);
        }
    /* vb, wb: adjoints of v1, w1 */
    /* ---- rows from the contacts */
    double Iib[9] = {0};
    for (int r = 0; r < nr; ++r) {
        const drow_t *D = &F->rows[r];
        if (!D->live) continue;
        drow_bar_t *X = &RBr[r];
        const body_t *B = &w->bodies[w->pairs[D->pair].b];
        double ab_[3][3], bb_[3][3], db_[3][3];
        memcpy(ab_, X->a, sizeof ab_);
        memcpy(bb_, X->b, sizeof bb_);
        memcpy(db_, X->d, sizeof db_);
        double rab[3] = {0, 0, 0}, uob[3] = {0, 0, 0}, rbb[3] = {0, 0, 0};
        for (int j = 0; j < 3; ++j) {
            const double denb = -D->k[j] * D->k[j] * X->k[j];      /* k = 1/den */
            invm_b += denb;
            for (int i = 0; i < 3; ++i) { ab_[j][i] += denb * D->b[j][i]; bb_[j][i] += denb * D->a[j][i]; }
            mv_vjp(F->Ii, D->a[j], bb_[j], ab_[j], Iib);           /* b = Ii a */
            for (int i = 0; i < 3; ++i) { uob[i] -= X->e[j] * D->d[j][i]; db_[j][i] -= X->e[j] * D->uo[i]; }
            cross_vjp(D->ra, D->d[j], ab_[j], rab, db_[j]);       /* a = ra x d */
        }
        mu_b[D->pair] += X->mu;
        double phib = X->bias * ((D->flags & 2) ? 1.0 / hs : w->cfg.baumgarte / hs);
        cross_vjp(B->w, D->rb, uob, NULL, rbb);                   /* uo = vB + wB x rb */
        double xbwb[3], xab[3], nbv[3];
        memcpy(xbwb, rbb, sizeof xbwb);                          /* rb = xbw - comB */
        memcpy(xab, rab, sizeof xab);                            /* ra = xa - com */
        for (int i = 0; i < 3; ++i) comb[i] -= rab[i];
        /* d0 = n, d1 = tr / |tr|, d2 = n x d1 */
        memcpy(nbv, db_[0], sizeof nbv);
        double d1b[3];
        memcpy(d1b, db_[1], sizeof d1b);
        cross_vjp(D->n, D->d[1], db_[2], nbv, d1b);
        const double dd = v_dot(D->d[1], d1b);
        double trb[3];
        for (int i = 0; i < 3; ++i) trb[i] = (d1b[i] - D->d[1][i] * dd) / D->tn;
        if (D->flags & 1) { nbv[2] += trb[1]; nbv[1] -= trb[2]; }
        else { nbv[2] -= trb[0]; nbv[0] += trb[2]; }
        /* xbw = xa - phi n */
        for (int i = 0; i < 3; ++i) { xab[i] += xbwb[i]; nbv[i] -= D->phi * xbwb[i]; }
        phib -= v_dot(D->n, xbwb);
        /* n = RB nb, nb = g / |g| */
        double RBm[9], RBt[9], nbb[3], gb[3], xblb[3], xwb[3];
        q_to_m(B->q, RBm);
        m_transpose(RBm, RBt);
        m_vec(RBt, nbv, nbb);
        const double gd = v_dot(D->nb, nbb);
        for (int i = 0; i < 3; ++i) gb[i] = (nbb[i] - D->nb[i] * gd) / D->gn;
        /* (phi, g) of the taped cell's trilinear polynomial at xbl */
        m_vec(D->H, gb, xblb);
        for (int i = 0; i < 3; ++i) xblb[i] += D->g[i] * phib;
        /* xbl = RB^T (xw - pB), xa = xw = R s + p */
        m_vec(RBm, xblb, xwb);
        v_add(xwb, xab, xwb);
        for (int i = 0; i < 3; ++i) {
            pbt[i] += xwb[i];
            for (int j = 0; j < 3; ++j) Rb[3 * i + j] += xwb[i] * D->s[j];
        }
    }
    free(lb);
    free(RBr);
    /* ---- external forces: v1 = v + hs (g + F/m), w1 = w + hs Ii (tau - w x Iw w) */
    *mass_b += -hs * v_dot(A->force, vb) / (m * m);
    double tqb[3], gyb[3], Lwb[3] = {0, 0, 0}, Iwb[9] = {0}, w0b[3];
    memcpy(w0b, wb, sizeof w0b);
    m_vec(F->Ii, wb, tqb);
    v_scale(tqb, hs, tqb);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Iib[3 * i + j] += hs * wb[i] * F->tq[j];
    v_scale(tqb, -1.0, gyb);
    cross_vjp(F->w0, F->Lw, gyb, w0b, Lwb);
    mv_vjp(F->Iw, F->w0, Lwb, w0b, Iwb);
    /* com = R com_b + p */
    for (int i = 0; i < 3; ++i) {
        pbt[i] += comb[i];
        for (int j = 0; j < 3; ++j) Rb[3 * i + j] += comb[i] * A->com_b[j];
    }
    /* Iw = R Ib R^T, Ii = R Ib^-1 R^T; Ib = m I_1, Ib^-1 = I_1^-1 / m, invm = 1/m */
    double Ibb[9] = {0}, Ibib[9] = {0};
    sandwich_vjp(F->R, A->Ib, Iwb, Rb, Ibb);
    sandwich_vjp(F->R, A->Ib_inv, Iib, Rb, Ibib);
    double s1 = 0, s2 = 0;
    for (int k = 0; k < 9; ++k) { s1 += Ibb[k] * A->Ib[k]; s2 += Ibib[k] * A->Ib_inv[k]; }
    *mass_b += s1 / m - s2 / m - invm_b / (m * m);
    q_to_m_vjp(F->q0, Rb, qb);
    memcpy(xb, pbt, 3 * sizeof(double));
    memcpy(xb + 3, qb, 4 * sizeof(double));
    memcpy(xb + 7, vb, 3 * sizeof(double));
    memcpy(xb + 10, w0b, 3 * sizeof(double));
}

/* ---- public entry points ---- */

int or_diff_record(or_world *w, int n_substeps, int n_iters) {
    if (w->cfg.n_vel_iters != 0 || w->cfg.solver != 0 || n_substeps < 1 || n_iters < 0) return -1;
    for (int e = 0; e < w->n_envs; ++e)
        if (diff_env_body(w, e) == -1) return -1;
    diff_tape_free(w);
    const double hs = w->cfg.dt / (double)n_substeps;
    w->tape = diff_tape_new(n_substeps, w->n_envs, n_iters, hs);
    for (int si = 0; si < n_substeps; ++si) {
        or_collide(w);
        for (int e = 0; e < w->n_envs; ++e) {
            dfwd_t F;
            diff_env_forward(w, e, si, 0, &F, 0);
            dfwd_free(&F);
        }
    }
    return 0;
}

int or_diff_replay(or_world *w) {
    if (!w->tape) return -1;
    for (int si = 0; si < w->tape->S; ++si)
        for (int e = 0; e < w->n_envs; ++e) {
            dfwd_t F;
            if (diff_env_forward(w, e, si, 1, &F, 0)) return -1;
            dfwd_free(&F);
        }
    return 0;
}

/* Gradient of a replay from the current state (which is left unchanged).  g_* are the
 * adjoints of the final state (n_bodies entries each); d_* receive those of the initial
 * state; d_mass (n_bodies) and d_mu (n_pairs) those of the parameters.  Bodies without
 * dynamics get zero. */
int or_diff_adjoint(or_world *w, const double *g_pos, const double *g_quat, const double *g_lin,
                    const double *g_ang, double *d_pos, double *d_quat, double *d_lin, double *d_ang,
                    double *d_mass, double *d_mu) {
    struct diff_tape *T = w->tape;
    if (!T) return -1;
    const int nb = w->n_bodies;
    double *x0 = (double *)malloc(sizeof(double) * 13 * nb);
    for (int i = 0; i < nb; ++i) {
        const body_t *b = &w->bodies[i];
        memcpy(x0 + 13 * i, b->p, 3 * sizeof(double)); memcpy(x0 + 13 * i + 3, b->q, 4 * sizeof(double));
        memcpy(x0 + 13 * i + 7, b->v, 3 * sizeof(double)); memcpy(x0 + 13 * i + 10, b->w, 3 * sizeof(double));
    }
    /* checkpoints: the state at each substep's start */
    double *ck = (double *)malloc(sizeof(double) * 13 * nb * (size_t)T->S);
    for (int si = 0; si < T->S; ++si) {
        for (int i = 0; i < nb; ++i) {
            const body_t *b = &w->bodies[i];
            double *c = ck + 13 * ((size_t)si * nb + i);
            memcpy(c, b->p, 3 * sizeof(double)); memcpy(c + 3, b->q, 4 * sizeof(double));
            memcpy(c + 7, b->v, 3 * sizeof(double)); memcpy(c + 10, b->w, 3 * sizeof(double));
        }
        for (int e = 0; e < w->n_envs; ++e) {
            dfwd_t F;
            diff_env_forward(w, e, si, 1, &F, 0);
            dfwd_free(&F);
        }
    }
    double *xb = (double *)calloc(13 * (size_t)nb, sizeof(double));
    for (int i = 0; i < nb; ++i) {
        memcpy(xb + 13 * i, g_pos + 3 * i, 3 * sizeof(double)); memcpy(xb + 13 * i + 3, g_quat + 4 * i, 4 * sizeof(double));
        memcpy(xb + 13 * i + 7, g_lin + 3 * i, 3 * sizeof(double)); memcpy(xb + 13 * i + 10, g_ang + 3 * i, 3 * sizeof(double));
    }
    for (int i = 0; i < nb; ++i) d_mass[i] = 0.0;
    for (int p = 0; p < w->n_pairs; ++p) d_mu[p] = 0.0;
    for (int si = T->S - 1; si >= 0; --si) {
        for (int i = 0; i < nb; ++i) {      /* recompute from the checkpoint */
            body_t *b = &w->bodies[i];
            const double *c = ck + 13 * ((size_t)si * nb + i);
            memcpy(b->p, c, 3 * sizeof(double)); memcpy(b->q, c + 3, 4 * sizeof(double));
            memcpy(b->v, c + 7, 3 * sizeof(double)); memcpy(b->w, c + 10, 3 * sizeof(double));
        }
        for (int e = 0; e < w->n_envs; ++e) {
            dfwd_t F;
            diff_env_forward(w, e, si, 1, &F, 1);
            if (F.ia >= 0) diff_env_reverse(w, &F, xb + 13 * F.ia, &d_mass[F.ia], d_mu);
            dfwd_free(&F);
        }
    }
    for (int i = 0; i < nb; ++i) {
        const int dyn = w->bodies[i].type == 2;
        for (int k = 0; k < 3; ++k) {
            d_pos[3 * i + k] = dyn ? xb[13 * i + k] : 0.0;
            d_lin[3 * i + k] = dyn ? xb[13 * i + 7 + k] : 0.0;
            d_ang[3 * i + k] = dyn ? xb[13 * i + 10 + k] : 0.0;
        }
        for (int k = 0; k < 4; ++k) d_quat[4 * i + k] = dyn ? xb[13 * i + 3 + k] : 0.0;
        body_t *b = &w->bodies[i];
        memcpy(b->p, x0 + 13 * i, 3 * sizeof(double)); memcpy(b->q, x0 + 13 * i + 3, 4 * sizeof(double));
        memcpy(b->v, x0 + 13 * i + 7, 3 * sizeof(double)); memcpy(b->w, x0 + 13 * i + 10, 3 * sizeof(double));
    }
    free(x0); free(ck); free(xb);
    return 0;
}

/* Tape exchange: sizes, then arrays in the layout described above. */
int or_diff_tape_info(const or_world *w, int *S, int *E, int *K, double *hs, int *n_contacts) {
    if (!w->tape) return -1;
    *S = w->tape->S; *E = w->tape->E; *K = w->tape->K; *hs = w->tape->hs; *n_contacts = w->tape->n_c;
    return 0;
}

int or_diff_get_tape(const or_world *w, int *c_off, int *c_rec, unsigned char *r_bits, unsigned char *b_bits) {
    const struct diff_tape *T = w->tape;
    if (!T) return -1;
    memcpy(c_off, T->c_off, sizeof(int) * ((size_t)T->S * T->E + 1));
    memcpy(c_rec, T->c_rec, sizeof(int) * 6 * (size_t)T->n_c);
    memcpy(r_bits, T->r_bits, (size_t)T->K * T->n_c);
    memcpy(b_bits, T->b_bits, (size_t)T->S * T->E);
    return 0;
}

int or_diff_set_tape(or_world *w, int S, int K, double hs, const int *c_off, const int *c_rec,
                     const unsigned char *r_bits, const unsigned char *b_bits) {
    if (S < 1 || K < 0 || w->cfg.n_vel_iters != 0) return -1;
    for (int e = 0; e < w->n_envs; ++e)
        if (diff_env_body(w, e) == -1) return -1;
    diff_tape_free(w);
    struct diff_tape *T = diff_tape_new(S, w->n_envs, K, hs);
    memcpy(T->c_off, c_off, sizeof(int) * ((size_t)S * w->n_envs + 1));
    T->n_c = T->cap_c = c_off[(size_t)S * w->n_envs];
    T->c_rec = (int *)malloc(sizeof(int) * 6 * (size_t)(T->n_c > 0 ? T->n_c : 1));
    T->r_bits = (unsigned char *)malloc((size_t)K * (T->n_c > 0 ? T->n_c : 1) + 1);
    memcpy(T->c_rec, c_rec, sizeof(int) * 6 * (size_t)T->n_c);
    memcpy(T->r_bits, r_bits, (size_t)K * T->n_c);
    memcpy(T->b_bits, b_bits, (size_t)S * w->n_envs);
    w->tape = T;
    return 0;
}

/* Parameters of the differentiable rollout: a dynamic body's mass (inertia scaled at
 * fixed geometry) and a pair's friction coefficient. */
int or_set_body_mass(or_world *w, int body, double mass) {
    if (body < 0 || body >= w->n_bodies || !(mass > 0.0)) return -1;
    body_t *b = &w->bodies[body];
    const double s = mass / b->mass;
    for (int k = 0; k < 9; ++k) { b->Ib[k] *= s; b->Ib_inv[k] /= s; }
    b->mass = mass;
    b->invm = (b->type == 2) ? 1.0 / mass : 0.0;
    return 0;
}

int or_set_pair_mu(or_world *w, int pair, double mu) {
    if (pair < 0 || pair >= w->n_pairs || !(mu >= 0.0)) return -1;
    w->pairs[pair].mu = mu;
    return 0;
}

int or_n_pairs(const or_world *w) { return w->n_pairs; }
double or_get_body_mass(const or_world *w, int body) { return w->bodies[body].mass; }
double or_get_pair_mu(const or_world *w, int pair) { return w->pairs[pair].mu; }
