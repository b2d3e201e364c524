/*
 * fw_oracle.h -- plain FP64 CPU oracle of the SDF contact substep.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code with the
 * CUDA path: the two are written separately from the paper (Factory, Sec. III) and
 * from the stated readings of the places where the paper is silent.
 *
 * Every routine is written for obviousness, not speed: brute-force loops, FP64
 * arithmetic, no blocking or reordering beyond what the definition states.
 *
 * What each part follows:
 *   - SDF definition and trilinear value/gradient .... Sec. III-A
 *   - SDF generation by sampling a triangle mesh ...... Sec. III-A; closest point on a
 *     triangle by the Voronoi-region test (Ericson, Real-Time Collision Detection
 *     5.1.5); inside/outside from the generalized winding number (Jacobson et al. 2013)
 *     with the Van Oosterom-Strackee solid angle
 *   - contact patches ................................. Sec. III-C, Algorithm 1
 *   - Gauss-Seidel contact solve with Coulomb friction,
 *     substepped integration ........................... Sec. III-B (cited solver);
 *     the update rule is the velocity-level projected Gauss-Seidel stated in
 *     fw_oracle.c
 *   - mass properties ................................. divergence theorem over the
 *     tetrahedra (origin, triangle)
 *
 * Parity status: every function here is pinned by a CPU test against closed forms,
 * invariants or brute force (tests/test_oracle_*.py), except the exact patch contents
 * of Algorithm 1 beyond the hand-derivable cases, which are pinned only by those
 * small cases and by the paper's contact-count band (Table "contact statistics").
 */
#ifndef FW_ORACLE_H
#define FW_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- geometry primitives ---- */
/* Closest point q on triangle (a,b,c) to p.  Returns the Voronoi region:
 * 0 face, 1/2/3 vertex a/b/c, 4 edge ab, 5 edge bc, 6 edge ca. */
int or_closest_point_triangle(const double p[3], const double a[3], const double b[3],
                              const double c[3], double q[3]);
/* Solid angle subtended at p by triangle (a,b,c), signed by orientation. */
double or_solid_angle(const double p[3], const double a[3], const double b[3], const double c[3]);
/* Generalized winding number of a closed mesh at p (1 inside, 0 outside). */
double or_winding_number(const double p[3], const float *V, const int *T, int nt);
/* Unsigned distance from p to the closest triangle. */
double or_point_mesh_distance(const double p[3], const float *V, const int *T, int nt);
/* Mass, centre of mass and inertia tensor about the centre of mass (row-major 3x3)
 * of the solid bounded by a closed outward-wound mesh of uniform density. */
void or_mass_properties(const float *V, const int *T, int nt, double density,
                        double *mass, double com[3], double inertia[9]);

/* ---- grids ---- */
/* Grid placement from the mesh bounding box (see fw_oracle.c, or_grid_params). */
void or_grid_params(const float *V, int nv, int res, float pad, int cubic,
                    float lo[3], float *h, int dims[3]);
/* Signed distance at grid nodes: phi = -(distance) inside, +(distance) outside.
 * nodes == NULL: all nodes, x fastest (idx = (k*ny + j)*nx + i). */
void or_bake_nodes(const float *V, const int *T, int nt, const float lo[3], float h,
                   const int dims[3], const long long *nodes, long long n_nodes,
                   double *phi, int n_threads);
/* Trilinear value and analytic gradient (grid frame).  valid[i] = 0 when the point is
 * outside the grid box (phi/grad then 0). */
void or_query_band(const double *grid, const float lo[3], float h, const int dims[3], float band_voxels,
                   const float *pts, int n, double *phi, double *grad, int *valid, int *n_stored, int *n_bricks);
void or_query(const double *grid, const float lo[3], float h, const int dims[3],
              const float *pts, int n, double *phi, double *grad, int *valid);

/* ---- simulation world ---- */
typedef struct {
    double gravity[3];
    double dt;
    double contact_offset;   /* candidate iff phi < contact_offset */
    double cos_patch;        /* normal similarity threshold for Assign / BinReduce */
    int max_patches;         /* N of the paper (128 <= N <= 256) */
    int batch_size;          /* points per Generate batch (paper: 1024) */
    double baumgarte;        /* bias factor for penetrating contacts */
    int n_vel_iters;         /* extra bias-free sweeps after integration */
    double max_angvel;       /* |omega| clamp at integration, 0 = off */
    double margin_len;       /* decision margin (m) below which a pair is not comparable */
    double margin_dot;       /* decision margin (dimensionless) */
    int n_threads;           /* OpenMP threads (0 = default) */
    int contact_gen;         /* 0: one candidate per surface sample; 1: one per triangle of
                                the point body's mesh, by local minimisation (R15) */
    int tri_iters;           /* steps of that minimisation */
    float sdf_band;          /* R17 narrow band in voxels (bricks of 8^3 cells); 0 = dense */
    int solver;              /* 0: Gauss-Seidel (R9); 1: weighted Jacobi (R18) */
} or_config;

typedef struct {             /* same layout as the ABI's fw_body_desc (104 bytes) */
    int asset;
    int type;                /* 0 static, 1 kinematic, 2 dynamic, 3 fixed axis */
    float mass;              /* <= 0: from density */
    float mu;
    float pos[3];
    float quat[4];           /* x, y, z, w */
    float linvel[3];
    float angvel[3];
    float axis[3];
    float force[3];
    float torque[3];
} or_body_desc;

typedef struct {
    int sample;              /* index of the point in the point body's sample list */
    int patch;               /* patch slot it was emitted from */
    double phi;
    double xa[3];            /* contact point on body A (world) */
    double xb[3];            /* xa - phi * n (world) */
    double n[3];             /* world normal, out of body B toward body A */
} or_contact;

typedef struct {             /* a reduction input (float: the same values a device gets) */
    int sample;
    float phi;
    float x[3];
    float n[3];
} or_candidate;

typedef struct or_world or_world;

or_world *or_create(const or_config *cfg);
void or_destroy(or_world *w);
/* OpenMP threads of the world's later calls (0 = the OpenMP default); test/timing use */
void or_set_threads(or_world *w, int n_threads);
int or_add_asset(or_world *w, const float *V, int nv, const int *T, int nt,
                 const float *samples, int ns, double density);
/* lazy = 1 bakes nodes only when a query first needs them. */
int or_asset_bake(or_world *w, int asset, int res, float pad, int cubic, int lazy);
int or_asset_set_grid(or_world *w, int asset, const float lo[3], float h, const int dims[3],
                      const float *values);
int or_asset_get_grid(const or_world *w, int asset, float lo[3], float *h, int dims[3]);
int or_asset_mass(const or_world *w, int asset, double *mass, double com[3], double inertia[9]);
/* n_pairs < 0: pile envs (R20), whose pairs a broad phase finds at every detection. */
int or_add_envs(or_world *w, int n_envs, const or_body_desc *bodies, int n_per_env,
                const int *pairs, int n_pairs);
int or_n_envs(const or_world *w);
int or_n_bodies(const or_world *w);
/* One frame (dt) of n_substeps substeps with n_iters sweeps each. */
int or_step(or_world *w, int n_substeps, int n_iters);
/* One substep of length hs; detect = 0 reuses the contacts currently stored. */
int or_substep(or_world *w, double hs, int n_iters, int detect);
/* Narrow phase of one pair at the current state, every sample of body a. */
int or_query_pair(or_world *w, int env, int pair, double *phi, double *nrm, int *valid,
                  double *gnorm);
/* The pair's candidates (phi < contact_offset) rounded to float, in sample order. */
int or_pair_candidates(or_world *w, int env, int pair, or_candidate *out, int cap, int *n_out);
/* Per triangle of the point body's mesh (R15), at the current poses: the minimiser on the
 * face (world), phi there, the world normal, valid (0: outside the grid or vanishing
 * gradient) and the smallest |phi_trial - phi| of the step decisions taken (the margin of
 * the result against rounding).  Arrays of n_tris (x3 for x, n). */
int or_tri_contacts(or_world *w, int env, int pair, double *x, double *phi, double *n, int *valid,
                    double *margin);
/* Contact detection + reduction at the current state. */
int or_collide(or_world *w);
int or_get_contacts(const or_world *w, int env, or_contact *out, int cap, int *n_out,
                    double *min_margin_len, double *min_margin_dot);
int or_set_contacts(or_world *w, int env, const or_contact *in, int n);
/* Contacts of one pair of an env (its list in sweep order), and a replacement of that
 * list alone (the env's other pairs keep theirs).  `pair` is the env-local pair index. */
int or_get_pair_contacts(const or_world *w, int env, int pair, or_contact *out, int cap, int *n_out);
int or_set_pair_contacts(or_world *w, int env, int pair, const or_contact *in, int n);
/* Per-env minimum decision margins over everything since the last reset. */
int or_env_margins(const or_world *w, int env, double *len, double *dot);
/* A pile env's current pairs (R20; from its last detection): (point body, SDF body) as
 * local body ids, in pair order, and each pair's colour in the last solve (-1: no contacts). */
int or_get_pile_pairs(const or_world *w, int env, int *ab, int *color, int cap, int *n_out);
/* One pair's smallest decision margins in its last detection (env-local pair index). */
int or_pair_margins(const or_world *w, int env, int pair, double *len, double *dot);
/* A pile env's pairs at the current poses (broad phase only; their contacts cleared). */
int or_find_pile_pairs(or_world *w, int env);
void or_reset_margins(or_world *w);
/* State arrays, n_bodies entries: pos 3, quat 4, linvel 3, angvel 3. */
int or_get_state(const or_world *w, double *pos, double *quat, double *linvel, double *angvel);
int or_set_state(or_world *w, const double *pos, const double *quat, const double *linvel,
                 const double *angvel);
/* Wall seconds spent so far in lazy SDF bakes (set-up work, excluded from step timing). */
double or_bake_seconds(const or_world *w);
/* Friction-cone record of the last solve: per contact row of env, (lambda_n, |lambda_t|, mu). */
int or_get_impulses(const or_world *w, int env, double *out, int cap, int *n_out);

/* ---- differentiable rollout (reverse mode with the discrete decisions held fixed) ----
 * Envs must have at most one dynamic body, the point body a of each of their pairs, with
 * static or kinematic partners, and n_vel_iters = 0.  See fw_oracle.c for the tape. */
/* One frame (dt) of n_substeps substeps with n_iters sweeps from the current state,
 * detection and decisions as in or_step, recording the tape; the state advances. */
int or_diff_record(or_world *w, int n_substeps, int n_iters);
/* The taped rollout from the current state with every decision taken from the tape. */
int or_diff_replay(or_world *w);
/* Reverse mode of or_diff_replay at the current state (left unchanged): adjoints of the
 * final state in, adjoints of the initial state, of each body's mass and of each pair's
 * friction coefficient out. */
int or_diff_adjoint(or_world *w, const double *g_pos, const double *g_quat, const double *g_lin,
                    const double *g_ang, double *d_pos, double *d_quat, double *d_lin, double *d_ang,
                    double *d_mass, double *d_mu);
int or_diff_tape_info(const or_world *w, int *S, int *E, int *K, double *hs, int *n_contacts);
int or_diff_get_tape(const or_world *w, int *c_off, int *c_rec, unsigned char *r_bits, unsigned char *b_bits);
int or_diff_set_tape(or_world *w, int S, int K, double hs, const int *c_off, const int *c_rec,
                     const unsigned char *r_bits, const unsigned char *b_bits);
int or_set_body_mass(or_world *w, int body, double mass);
int or_set_pair_mu(or_world *w, int pair, double mu);
int or_n_pairs(const or_world *w);
double or_get_body_mass(const or_world *w, int body);
double or_get_pair_mu(const or_world *w, int pair);

/* Algorithm 1 on a given candidate list (sorted by sample index is not required). */
int or_reduce(const or_candidate *cand, int n, double cos_patch, int max_patches,
              int batch_size, or_contact *out, int cap, int *n_out, int *n_patches,
              double *min_margin_len, double *min_margin_dot);

#ifdef __cplusplus
}
#endif
#endif
