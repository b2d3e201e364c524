/*
 * fw.h -- C ABI of libfw, a single-GPU (sm_103a) implementation of the batched
 * contact-simulation substep of Factory (Narang et al., arXiv 2205.03532, Sec. III):
 *
 *   (a) SDF narrow phase: surface sample points of one body are transformed into the
 *       other body's frame and looked up in its voxel signed-distance field
 *       (trilinear value + gradient), Sec. III-A;
 *   (b) contact reduction of the candidates into normal-similar patches,
 *       Sec. III-C and Algorithm 1;
 *   (c) a Gauss-Seidel contact solve with Coulomb friction and substepped
 *       integration, Sec. III-B (the paper cites the solver; the update rule used here
 *       is stated at fw_step).
 *
 * Conventions for every call:
 *   - Units are SI (metres, seconds, kilograms).  Quaternions are (x, y, z, w).
 *   - Every input array is COPIED; the caller keeps ownership of its buffers.
 *   - Output arrays are caller-owned.  Where a call takes `device_ptrs`, 0 means host
 *     pointers and 1 means device pointers (for example torch CUDA tensors) on the
 *     world's device.
 *   - Nothing throws across the ABI.  Every call returns an fw_status; on failure
 *     fw_last_error() holds a message.  A NULL world returns FW_ERR_ARG.
 *   - A world is used by one host thread at a time.  GPU work is enqueued on the
 *     world's stream (fw_config.cuda_stream, or a stream the world creates) and is
 *     stream-ordered; calls that return data to host memory synchronise that stream.
 *   - Device-side problems (non-finite state, a contact buffer overflow) set a status
 *     word on the device; fw_sync() and every synchronising call report it.
 */
#ifndef FW_H
#define FW_H

#if defined(__GNUC__)
#define FW_API __attribute__((visibility("default")))
#else
#define FW_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fw_world fw_world;   /* opaque; owned by the library */

typedef enum {
    FW_OK = 0,
    FW_ERR_ARG = -1,            /* bad argument (NULL pointer, size, id out of range) */
    FW_ERR_OOM = -2,            /* device or host allocation failed */
    FW_ERR_CUDA = -3,           /* a CUDA runtime call failed (message in fw_last_error) */
    FW_ERR_STATE = -4,          /* call out of order (e.g. SDF body without a baked SDF) */
    FW_ERR_NONFINITE = -5,      /* a body state became NaN/Inf on the device */
    FW_ERR_OVERFLOW = -6,       /* an output buffer was too small */
    FW_ERR_TIMEOUT = -7,        /* a bounded device wait gave up */
    FW_ERR_DEVICE_BOUNDS = -8   /* a device-side index check failed */
} fw_status;

typedef enum {
    FW_BODY_STATIC = 0,         /* never moves; infinite mass */
    FW_BODY_KINEMATIC = 1,      /* moves with its prescribed linvel/angvel; infinite mass */
    FW_BODY_DYNAMIC = 2,        /* free rigid body */
    FW_BODY_FIXED_AXIS = 3      /* centre of mass fixed; spins about `axis` only (gears) */
} fw_body_type;

/* Simulation constants.  The paper states none of these except the frame time and the
 * batch size; the defaults are this library's readings (fw_config_default). */
typedef struct {
    float gravity[3];           /* m/s^2, default (0, 0, -9.81) */
    float dt;                   /* frame time, default 1/60 s (Table perf caption) */
    float contact_offset;       /* candidate iff phi < contact_offset; default 1e-4 m */
    float cos_patch;            /* normal similarity for Assign/BinReduce; default 0.94 */
    int max_patches;            /* N of Sec. III-C (128 <= N <= 256); default 128 */
    int patch_dirs;             /* direction slots per patch (beside the deepest); must be 6 */
    int batch_size;             /* samples per Generate batch; must be 1024 (Sec. III-C) */
    float baumgarte;            /* bias factor for penetrating contacts; default 0.2 */
    int n_vel_iters;            /* bias-free sweeps after integration; default 0 */
    float max_angvel;           /* |omega| clamp at integration, 0 = off; default 0 */
    int sdf_fp16;               /* 1: look up FP16 copies of the grids (phi/h); default 0 */
    int contact_gen;            /* 0: one candidate per surface sample of the point body
                                   (default); 1: one per triangle of its mesh, the minimiser
                                   of the SDF over the face by projected gradient descent
                                   with adaptive steps (Sec. III-A); Generate batches are
                                   then 1024 triangles and a contact's `sample` is the
                                   triangle index */
    int tri_iters;              /* descent steps per triangle (contact_gen = 1); default 16 */
    float sdf_band;             /* narrow-band bricked SDF storage, band half-width in voxels;
                                   0 (default): dense cell-corner copies.  Cells are grouped in
                                   bricks of 8^3; a brick is kept when a node of its cells has
                                   |phi| <= sdf_band * h or its nodes change sign, and a lookup
                                   in a brick left out answers phi = +band (-band inside) with a
                                   zero gradient, i.e. no candidate.  Every point with |phi| <=
                                   band reads exactly the dense value (sparse SDF storage,
                                   which the paper's Limitations section plans against the
                                   grids' memory footprint) */
    int solver;                 /* 0 (default): projected Gauss-Seidel; 1: weighted Jacobi --
                                   per sweep every contact's block update (normal row, then
                                   friction rows with its own normal change, disk projection)
                                   from the sweep-start velocities, all taken with weight
                                   1 / (contacts that can act); envs with at most one movable
                                   body; no adjoint (the solver the paper's solver comparison
                                   sizes at 8 substeps x 64 iterations) */
    int device;                 /* CUDA device ordinal, default 0 */
    void *cuda_stream;          /* cudaStream_t to enqueue on, NULL: the world's own */
    unsigned long long seed;    /* the seed the caller's scene generator drew its inputs
                                   with, kept with the world for its records; no step of
                                   the path draws a random number (poses, samples and
                                   masses are inputs), so nothing reads it; default 0 */
} fw_config;

/* One body of an environment.  104 bytes, no padding. */
typedef struct {
    int asset;                  /* asset id from fw_add_mesh_asset */
    int type;                   /* fw_body_type */
    float mass;                 /* kg; <= 0: from the asset's density (inertia scales) */
    float mu;                   /* friction coefficient; a pair uses sqrt(mu_a mu_b) */
    float pos[3];               /* world position of the asset frame */
    float quat[4];              /* world orientation of the asset frame (x, y, z, w) */
    float linvel[3];            /* centre-of-mass velocity */
    float angvel[3];            /* angular velocity (world) */
    float axis[3];              /* FIXED_AXIS: world spin axis */
    float force[3];             /* constant applied force at the centre of mass */
    float torque[3];            /* constant applied torque (world) */
} fw_body_desc;

/* A reduced contact as returned to callers.  52 bytes. */
typedef struct {
    int sample;                 /* index of the point in the point body's sample list */
    int patch;                  /* patch slot the contact came from */
    int pair;                   /* pair index within its environment */
    float phi;                  /* signed distance of the sample from body B (m) */
    float xa[3];                /* contact point on body A (world) */
    float xb[3];                /* xa - phi * n (world) */
    float n[3];                 /* unit normal out of body B toward body A (world) */
} fw_contact;

/* A reduction input for fw_reduce.  32 bytes. */
typedef struct {
    int sample;
    float phi;
    float x[3];
    float n[3];
} fw_candidate;

/* ---------------------------------------------------------------- world lifetime */

/* Fills *cfg with the defaults listed in fw_config. */
FW_API void fw_config_default(fw_config *cfg);

/* Creates a world on cfg->device: the container of many independent environments that are
 * stepped in parallel on one GPU (Sec. III-D runs 1,024 of them), with the simulation
 * constants of fw_config (frame time 1/60 s and substeps per frame: the caption of Table
 * "performance statistics"; Generate batches of 1024 and N patches per pair: Sec. III-C).
 * *out receives the handle (NULL on failure).
 * Errors: FW_ERR_ARG for batch_size != 1024, patch_dirs != 6, max_patches outside 1..256,
 * dt <= 0. */
FW_API fw_status fw_create(const fw_config *cfg, fw_world **out);

/* Frees every device and host resource of the world (no counterpart in the paper).  NULL
 * is accepted. */
FW_API fw_status fw_destroy(fw_world *w);

/* ---------------------------------------------------------------- assets */

/* Adds a closed, outward-wound triangle mesh (verts n_verts x 3, tris n_tris x 3, both
 * row-major host arrays).  sample_pts (n_samples x 3, asset frame, may be NULL when the
 * asset is only ever an SDF body) are the points queried against other bodies' SDFs
 * (Sec. II-A1 and III-A: surface points of the mesh body are tested against the SDF of
 * the other body); their order defines the sample index and the Generate batches of
 * Algorithm 1.  Mass, centre of mass and inertia come from the divergence theorem at
 * `density` (kg/m^3).  Errors: FW_ERR_ARG for bad sizes, n_samples > 2^24, or a mesh
 * enclosing no volume. */
FW_API fw_status fw_add_mesh_asset(fw_world *w, const float *verts, int n_verts, const int *tris,
                                   int n_tris, const float *sample_pts, int n_samples,
                                   float density, int *asset_id_out);

/* Bakes the asset's SDF on the GPU once, at set-up (Sec. III-A: the SDF is sampled from
 * the triangle mesh when the object is created).  Node-centred grid over the box padded
 * by padding_m; `resolution` nodes along the longest padded axis (the per-asset SDF
 * resolution of the appendix on using the contact methods); cubic = 1 gives
 * resolution^3 nodes.  h, lo are float32: h = fl(L / (res - 1)),
 * lo_a = fl(centre_a - h (dims_a - 1) / 2).  Value at a node: -(distance) inside the
 * solid, +(distance) outside; distance to the closest triangle found in float32 and
 * re-evaluated in float64, sign from the closest feature's angle-weighted pseudonormal
 * (float64 winding number where that test is ambiguous).  Synchronous.
 * Errors: FW_ERR_ARG (resolution < 2), FW_ERR_OOM. */
FW_API fw_status fw_bake_sdf(fw_world *w, int asset_id, int resolution, float padding_m, int cubic);

/* Installs a caller-made SDF grid instead of baking (values: host, dims[2] x dims[1] x
 * dims[0], x fastest).  Used to test the lookup on exactly known grids. */
FW_API fw_status fw_set_sdf(fw_world *w, int asset_id, const float lo[3], float h,
                            const int dims[3], const float *values);

/* Reads back the grid placement and, if values != NULL, the float32 node values (host
 * array of dims product). */
FW_API fw_status fw_get_sdf(fw_world *w, int asset_id, float lo[3], float *h, int dims[3],
                            float *values);

/* Mass properties used for the asset (density based): mass, centre of mass (asset
 * frame) and inertia about it (row-major 3x3), host arrays. */
/* Device bytes of an asset's SDF lookup copy (the cell-corner copy, dense or bricked,
 * plus the brick table) and, with narrow-band storage, the bricks kept and the bricks of
 * the grid (both 0 when dense).  FW_ERR_STATE when the asset has no SDF.  Any pointer may
 * be NULL. */
FW_API fw_status fw_get_sdf_storage(fw_world *w, int asset_id, long long *cell_bytes, int *bricks_stored,
                                    int *bricks_total);
FW_API fw_status fw_get_mass(fw_world *w, int asset_id, double *mass, double com[3],
                             double inertia[9]);

/* ---------------------------------------------------------------- environments */

/* Adds n_envs environments of n_per_env bodies each (per_env: n_envs x n_per_env
 * descriptors, env-major; 1..8 bodies) and n_pairs contact pairs per environment
 * (pairs: n_pairs x 2 local body ids (a, b), 0..63 pairs); a is queried with its sample
 * points against b's SDF (appendix on using the contact methods: the body with the
 * SDF is queried by the other body's mesh).  Envs are independent.  May be called
 * several times with different structures (uneven batches).  *first_env_out receives
 * the id of the first new env.  Errors: FW_ERR_STATE if a b body's asset has no SDF or
 * an a body's asset has no samples; FW_ERR_ARG for bad ids or sizes. */
FW_API fw_status fw_add_env_bodies(fw_world *w, int n_envs, const fw_body_desc *per_env,
                                   int n_per_env, const int *pairs, int n_pairs,
                                   int *first_env_out);

/* Adds one pile environment: n_bodies bodies (1..1024; host descriptors) in one scene, the
 * scenes of the paper's experiments where 1024 nuts, bowls or toruses fall into a pile in
 * one environment (Sec. III-D, scene list; Table "contact statistics", row Nuts).  Its pairs are
 * not listed: every detection finds them again (pair finding, part of contact handling in
 * that table) -- for local bodies i < j, at least one of them dynamic or fixed-axis, i's
 * samples against j's SDF when i has samples and j an SDF, else j's samples against i's
 * SDF when j has samples and i an SDF, and only when the bodies' bounding spheres (about
 * their asset origins) are within the contact offset plus two voxels of the SDF body's
 * grid (no sample can have a candidate farther apart); pairs in (i, j) order.  Each pair's
 * contacts come from the same narrow phase and Algorithm 1 as a listed pair's.  The solve
 * (Sec. III-B) colours the pairs that have contacts greedily in pair order (each takes the
 * lowest of 64 colours that no earlier pair sharing one of its movable bodies took; the
 * last colour gathers the rest) and sweeps colour by colour, pair order within a colour:
 * the same updates as one Gauss-Seidel sweep over the rows in that order.
 * max_pairs, max_contacts: capacities of the pile's pair list (at most 65535) and of its
 * contact rows (below 2^21) (0: 8 pairs and 192 contacts per body); pairs or rows beyond
 * them are dropped and the next synchronising call returns FW_ERR_OVERFLOW.  Piles need contact_gen = 0 and the
 * Gauss-Seidel solver, and are not differentiable (fw_record_rollout refuses them).
 * *env_out receives the env id.  Errors: FW_ERR_ARG for bad sizes or descriptors, or a pile
 * too large for the solve's shared memory (73 n_bodies + 11 max_pairs bytes); FW_ERR_STATE
 * when a movable body's asset has neither samples nor an SDF. */
FW_API fw_status fw_add_pile(fw_world *w, const fw_body_desc *bodies, int n_bodies, int max_pairs,
                             int max_contacts, int *env_out);

/* A pile env's current pairs (those of its last detection): pairs n x 2 local body ids
 * (sample body, SDF body) in pair order, and if colors != NULL each pair's colour in the
 * last solve (-1: no contacts, or no solve since the detection).  Host arrays of cap
 * entries; synchronises.  *n_out receives the pair count; FW_ERR_OVERFLOW when it is more
 * than cap.  The `pair` index of fw_get_contacts / fw_set_contacts for a pile env is this
 * pair order.  Errors: FW_ERR_ARG when env is not a pile env. */
FW_API fw_status fw_get_pile_pairs(fw_world *w, int env, int *pairs, int *colors, int cap, int *n_out);

/* ---------------------------------------------------------------- stepping */

/* Advances every environment by one frame dt as n_substeps substeps of
 * hs = dt / n_substeps (substeps and solver iterations per frame: Sec. III-B and Table
 * "performance statistics"; the substep itself: Sec. III-A SDF collisions, Sec. III-C
 * contact reduction, Sec. III-B solve).  Each substep: external forces (gravity, applied force and
 * torque, gyroscopic term); contact detection and reduction at the current poses;
 * constraint rows per contact (normal, two tangents, effective masses, bias
 * phi/hs if phi > 0 else baumgarte*phi/hs); n_iters Gauss-Seidel sweeps, each contact's
 * normal impulse clamped to >= 0 and then its two friction impulses projected jointly
 * on the disk of radius mu * normal impulse; semi-implicit Euler integration of the
 * centre of mass and q <- normalize(q + hs/2 (omega,0) q); n_vel_iters bias-free sweeps.
 * Enqueued as one CUDA graph (captured on first use for a given (n_substeps, n_iters)
 * and topology); does not synchronise.
 * Errors: FW_ERR_ARG for n_substeps < 1 or n_iters < 0. */
FW_API fw_status fw_step(fw_world *w, int n_substeps, int n_iters);

/* One substep of length hs.  detect = 0 reuses the contacts now in the contact buffer
 * (from fw_collide or fw_set_contacts).  Enqueued; does not synchronise. */
FW_API fw_status fw_substep(fw_world *w, float hs, int n_iters, int detect);

/* Contact detection and reduction at the current poses, into the contact buffer. */
FW_API fw_status fw_collide(fw_world *w);

/* Contacts of one env from the contact buffer, pairs in order (host array; synchronises).
 * Errors: FW_ERR_OVERFLOW when more than cap (n_out still receives the count). */
FW_API fw_status fw_get_contacts(fw_world *w, int env, fw_contact *out, int cap, int *n_out);

/* Replaces the contacts of one env (host array; `pair` selects the pair of each one;
 * the contacts of a pair must be contiguous and in sweep order).  For solving given
 * contacts with fw_substep(detect = 0).  A pile env keeps the pairs of its last detection
 * (fw_get_pile_pairs); `pair` indexes them. */
FW_API fw_status fw_set_contacts(fw_world *w, int env, const fw_contact *in, int n);

/* ---------------------------------------------------------------- state */

/* Body state of all bodies (global body order = env order, then body order; see
 * fw_get_env_info): pos n x 3, quat n x 4, linvel n x 3, angvel n x 3 (float32) -- the
 * state the integration of Sec. III-B advances, and all a frame needs to resume (contacts
 * are detected again every substep and impulses start at zero).  Any pointer may be NULL
 * to skip it.  device_ptrs = 0 synchronises. */
FW_API fw_status fw_get_state(fw_world *w, float *pos, float *quat, float *linvel,
                              float *angvel, int device_ptrs);
/* Sets the state of Sec. III-B's integration (the layout of fw_get_state); quaternions are
 * normalised on the device.  device_ptrs = 0 synchronises before returning so host buffers
 * may be reused. */
FW_API fw_status fw_set_state(fw_world *w, const float *pos, const float *quat,
                              const float *linvel, const float *angvel, int device_ptrs);

/* ---------------------------------------------------------------- test hooks */

/* Trilinear SDF value and gradient of an asset's grid at n points given in the asset
 * frame (Sec. III-A); phi n, grad n x 3.  Points outside the grid give phi = +inf and
 * grad = 0.  Synchronises when device_ptrs = 0. */
FW_API fw_status fw_query_sdf(fw_world *w, int asset_id, const float *pts, int n, float *phi,
                              float *grad, int device_ptrs);

/* Per-triangle contact generation of one pair at the current poses (contact_gen = 1's
 * Generate step, whatever the world's contact_gen): for each triangle of the point body's
 * mesh, the minimiser of body B's SDF over the face by projected gradient descent with
 * adaptive steps, tri_iters steps (Sec. III-A; centroid start, first step half the
 * longest edge, accepted steps grow by 1.5, rejected ones halve, closest-point
 * projection onto the face).  Outputs per triangle (n_tris entries): x (3 floats, world)
 * the minimiser on the face, phi there (+inf when the centroid lies outside B's grid or
 * the gradient vanishes), normal (3 floats, world, the unit SDF gradient).  Host or
 * device arrays per device_ptrs; synchronises for host arrays. */
FW_API fw_status fw_tri_contacts(fw_world *w, int env, int pair, float *x, float *phi, float *normal,
                                 int device_ptrs);

/* The narrow phase of one pair at the current poses, for every sample point of body a:
 * phi (n_samples) and the world normal (n_samples x 3); phi = +inf where the point is
 * outside the grid or the gradient vanishes.  Same device code as the step. */
FW_API fw_status fw_query_pair(fw_world *w, int env, int pair, float *phi, float *normal,
                               int device_ptrs);

/* Algorithm 1 on a caller-given candidate list (host array, any order, unique samples)
 * with the world's cos_patch and max_patches: the same device code as the step's
 * reduction.  Outputs contacts (host, pair = 0) and the number of patches. */
FW_API fw_status fw_reduce(fw_world *w, const fw_candidate *cands, int n, fw_contact *out,
                           int cap, int *n_out, int *n_patches);

/* Algorithm 1 on candidates already in device memory, without allocating anything.
 * The paper has no counterpart to this call; it exists for callers that must not
 * allocate device memory once they are running -- for example a control loop with a
 * fixed latency budget (cudaMalloc and cudaFree can stall the whole device), or a host
 * program whose memory pool owns the GPU (PyTorch's caching allocator) and lets no one
 * else allocate.  On candidates sorted by sample it runs the same reduction code as
 * fw_reduce and returns the same contacts and patch count; it differs in how it reports
 * problems: an overflow (more contacts than cap) is reported through d_counts[0] > cap,
 * not through a status, and the input must already be sorted (fw_reduce sorts a copy).
 *   d_cands   device array of n candidates, samples strictly increasing and < 65536
 *             (the limit of the call's fixed scratch), n <= 65536;
 *   d_out     device array for up to cap contacts (fw_contact, pair = 0); nothing is
 *             written past entry cap - 1;
 *   d_counts  device int[2]: number of contacts (may exceed cap; only cap are written)
 *             and number of patches; (-1, 0) when the device finds the candidates
 *             unsorted, repeated or out of range.
 * Scratch: one 2.2 MB block of device memory that every GPU loading the library holds
 * until the process exits, shared by all calls and keeping the last call's contents
 * (nothing in it needs to start at zero).  Calls that overlap on the GPU (two streams, two
 * worlds) race on it: order them on one stream.  The first call on a device (from any
 * host thread; concurrent first calls are serialised) looks the block's address up, with
 * no allocation; make that first call before any stream capture.  The address is kept for
 * the life of the process: a program that resets the device (cudaDeviceReset) must not
 * call this function afterwards.
 * Enqueued on the world's stream, which must be ordered after the writes of d_cands and
 * d_counts' previous readers; does not synchronise.
 * Errors: FW_ERR_ARG for NULL pointers or n > 65536 (a clear message in fw_last_error). */
FW_API fw_status fw_reduce_noalloc(fw_world *w, const fw_candidate *d_cands, int n, fw_contact *d_out,
                                   int cap, int *d_counts);

/* ------------------------------------------------ differentiable rollout */
/* Reverse mode of the substep with its discrete decisions held fixed (no counterpart in
 * the paper, which simulates forward only).  Envs taking part have at most one dynamic
 * body, the point-sampled body a of each of their pairs, with static or kinematic
 * partners (no fixed-axis bodies), and the world has n_vel_iters = 0 and contact_gen = 0
 * (per-sample contacts: the tape rebuilds every contact from its surface sample, which a
 * per-triangle contact does not have; such worlds are refused with FW_ERR_ARG before
 * anything is enqueued).
 *
 * fw_record_rollout: one frame (dt) of n_substeps substeps with n_iters Gauss-Seidel
 * sweeps from the current state, each substep running detection (Sec. III-A, III-C) and
 * then the differentiable solve (Sec. III-B: normal row with lambda_n >= 0, friction rows
 * projected jointly on the disk, semi-implicit integration), recording a tape of every
 * discrete decision: the contacts (sample, pair, SDF cell), the tangent and bias
 * branches, per contact and sweep the normal clamp and friction projection, and the
 * |omega| clamp; and a checkpoint of the state at each substep's start.  The state
 * advances.  FW_ERR_ARG when an env does not qualify.  Device memory for the tape and
 * the checkpoints is allocated here (freed by the next record or fw_destroy).
 * fw_replay_rollout: the recorded rollout again from the current state with every
 * decision taken from the tape (the taped cell's trilinear polynomial is used even a
 * little outside it): a smooth function of the initial state, the dynamic bodies'
 * masses and the pairs' friction coefficients, equal to the recorded forward at the
 * recorded point.  Writes new checkpoints.  FW_ERR_STATE without a record.
 * fw_adjoint_rollout: the reverse mode of that function at the initial state of the
 * last record or replay: given the adjoints of the final state (g_*, n_bodies entries
 * of 3/4/3/3 floats), returns the adjoints of the initial state (d_*), of each body's
 * mass (d_mass, n_bodies; inertia scales with mass at fixed geometry) and of each
 * pair's friction coefficient (d_mu, n_pairs).  Bodies that are not dynamic get zero.
 * Each substep is recomputed from its checkpoint, last first.  device_ptrs selects host
 * (0) or device (1) arrays.  Synchronises.
 * fw_get_tape: info = (substeps, envs, sweeps, contacts); with non-NULL arrays also the
 * tape: c_off (substeps*envs + 1 offsets, env-major within each substep), c_rec (6 ints
 * per contact: sample, pair, cell i, j, k, flags bit 0 t1 from n x e_x, bit 1 phi > 0),
 * r_bits (sweeps per contact: bit 0 lambda_n > 0 after the row, bit 1 projected),
 * b_bits (substeps*envs: bit 0 |omega| clamped).  Synchronises.
 * fw_set_body_params: mass (n_bodies, <= 0 keeps; inertia rescaled with the mass) and
 * mu (n_pairs, < 0 keeps), host arrays, either may be NULL.  Synchronises. */
FW_API fw_status fw_record_rollout(fw_world *w, int n_substeps, int n_iters);
FW_API fw_status fw_replay_rollout(fw_world *w);
FW_API fw_status fw_adjoint_rollout(fw_world *w, const float *g_pos, const float *g_quat, const float *g_linvel,
                                   const float *g_angvel, float *d_pos, float *d_quat, float *d_linvel,
                                   float *d_angvel, float *d_mass, float *d_mu, int device_ptrs);
/* The same two operations under the names of the frame-step interface:
 * fw_step_fwd_ckpt(w, n_substeps, n_iters) is fw_record_rollout: one frame forward with
 * its tape and per-substep checkpoints; fw_step_bwd(w, ...) is fw_adjoint_rollout of the
 * frame last recorded (or replayed).  Arguments, ownership and errors as there. */
FW_API fw_status fw_step_fwd_ckpt(fw_world *w, int n_substeps, int n_iters);
FW_API fw_status fw_step_bwd(fw_world *w, const float *g_pos, const float *g_quat, const float *g_linvel,
                             const float *g_angvel, float *d_pos, float *d_quat, float *d_linvel, float *d_angvel,
                             float *d_mass, float *d_mu, int device_ptrs);
FW_API fw_status fw_get_tape(fw_world *w, int info[4], int *c_off, int *c_rec, unsigned char *r_bits,
                             unsigned char *b_bits);
FW_API fw_status fw_set_body_params(fw_world *w, const float *mass, const float *mu);

/* ---------------------------------------------------------------- diagnostics */

/* Waits for the world's stream and reports the device status word. */
FW_API fw_status fw_sync(fw_world *w);

/* Per-kernel timing.  enable = 1 makes later fw_step calls launch their kernels
 * directly (no graph) with a CUDA event pair around each launch; fw_get_timings then
 * synchronises and returns, summed over the launches since the previous call:
 * ms[0] detection ms (query + reduction kernels), ms[1] solve + integration kernel ms,
 * ms[2] number of detection passes, ms[3] number of solve launches (n >= 4), and when
 * n > 4: ms[4] query kernel ms, ms[5] reduction kernel ms; further entries are 0. */
FW_API fw_status fw_set_timing(fw_world *w, int enable);
FW_API fw_status fw_get_timings(fw_world *w, float *ms, int n);

/* Launch shape of the solve kernel.  envs_per_warp in {1, 2, 4, 8}: that many environments
 * share one warp, each on 32 / envs_per_warp lanes (fewer, longer-lived warps when the
 * env count exceeds the device's schedulers); warps_per_block in 1..4.  0 for either
 * lets the library choose from the env count and the device (the default).  A value that
 * does not fit the device's shared memory for this world is lowered when launching.
 * Results do not depend on the shape (each env runs the same arithmetic in any lane
 * group).  Errors: FW_ERR_ARG for values outside those sets.  fw_get_solve_shape returns
 * the shape the next fw_step will launch. */
FW_API fw_status fw_set_solve_shape(fw_world *w, int envs_per_warp, int warps_per_block);
/* Autotuner of that shape: at the current state, runs detection once for n_substeps /
 * n_iters, then times `trials` solve launches for every shape that fits (envs per warp
 * 1, 2, 4, 8 x warps per block 1..4), restoring the body state before each, and keeps
 * the fastest (as fw_set_solve_shape would; a shape tried later must beat the best so far
 * by more than 1%).  The state is left as it was.  Returns the
 * chosen shape and its time per solve launch (ms); any output pointer may be NULL.
 * Allocates and frees one state-sized device buffer; synchronises. */
FW_API fw_status fw_autotune_solve(fw_world *w, int n_substeps, int n_iters, int trials, int *envs_per_warp,
                                   int *warps_per_block, float *best_ms);
FW_API fw_status fw_get_solve_shape(fw_world *w, int *envs_per_warp, int *warps_per_block);

/* Launch shape of detection (Sec. III-A narrow phase, Sec. III-C Algorithm 1):
 * query_threads in {128, 256, 512} threads per work item of 1024 samples (each thread
 * queries 1024 / query_threads samples; per-triangle generation always runs 256) and
 * reduce_warps in {2, 4, 8} warps per pair; 0 for either: the default (256, 4).  Results
 * do not depend on the shape: candidates are compacted in sample order and the reduction
 * breaks every tie by depth and sample.  Errors: FW_ERR_ARG for other values.
 * fw_get_detect_shape returns the shape in use. */
FW_API fw_status fw_set_detect_shape(fw_world *w, int query_threads, int reduce_warps);

/* The narrow phase's cull (Sec. III-A; on by default): each warp's 32 consecutive sample
 * points (the samples an asset is given sorted along a space-filling curve stay close)
 * lie in a bounding sphere computed when the asset is added; when the sphere lies outside
 * the other body's grid box, or that body's SDF at the sphere's centre exceeds the contact
 * offset by more than the interpolated field can change over the radius (2.5 x radius, an
 * interpolated distance field changing by at most sqrt(3) per unit length, plus FP16
 * rounding, plus one voxel), none of the 32 can be a candidate and their lookups are
 * skipped.  Dense SDF storage only.  The candidates, and
 * everything after them, are the same with the cull on or off.  on: 1 or 0; errors:
 * FW_ERR_ARG for other values.  fw_get_query_cull writes 1 or 0 to *on (the setting in use,
 * which fw_autotune_detect may have changed). */
FW_API fw_status fw_set_query_cull(fw_world *w, int on);
FW_API fw_status fw_get_query_cull(fw_world *w, int *on);

/* Test hook of failure detection (no counterpart in the paper): makes one of the kernels'
 * bounded device waits run out, as a lost copy or a missing block would.  what = 1: every
 * grid barrier of the pile sweep kernel waits for one more block than the launch has;
 * what = 2: the fast solve's row stream issues no chunk copy, so the waits for its chunks
 * see no arrival.  Each wait gives up after a bounded number of polls (about a second for a
 * grid barrier, tens of milliseconds for a chunk), sets the timeout status and the
 * kernel ends (its results are then meaningless); the next synchronising call returns
 * FW_ERR_TIMEOUT and the world stays usable.  0 (default) turns it off. */
FW_API fw_status fw_test_stall(fw_world *w, int what);
FW_API fw_status fw_get_detect_shape(fw_world *w, int *query_threads, int *reduce_warps);
/* Autotuner of that shape: at the current poses, runs one detection, then times `trials`
 * query launches for each query size (with 4 reduction warps), and `trials` reduction
 * launches of the fastest query's candidates for each warp count, and keeps the fastest of
 * each (as fw_set_detect_shape would; the default is tried first and another shape must
 * beat it by more than 1%).  Between the two it times the chosen query with the cull
 * (fw_set_query_cull) on and off and keeps it on only when that is faster by more than 10%
 * (what the cull saves can shrink as bodies come together; its cost does not).
 * Every timed configuration first runs one untimed pass (its kernels' first launch loads
 * their module).  The body state is not touched; the contact buffer
 * is left holding the contacts at the current poses.  Returns the chosen shape and the
 * summed time of one query and one reduction launch (ms); any output pointer may be NULL.
 * Synchronises. */
FW_API fw_status fw_autotune_detect(fw_world *w, int trials, int *query_threads, int *reduce_warps,
                                    float *best_ms);

/* Totals of the last detection pass (synchronises): candidates (samples with phi below
 * the contact offset, Sec. III-A) summed over all pairs, and reduced contacts kept
 * (Algorithm 1) summed over all pairs.  Either pointer may be NULL.  Counts are those of
 * the most recent substep that ran detection (0 before any). */
FW_API fw_status fw_get_detect_stats(fw_world *w, long long *n_candidates, long long *n_contacts);

/* Sizes: n_envs, n_bodies, n_pairs (any pointer may be NULL). */
FW_API fw_status fw_get_counts(fw_world *w, int *n_envs, int *n_bodies, int *n_pairs);

/* Where one environment's bodies and pairs sit in the world's global order (the index of its
 * first body in fw_get_state's arrays, its body count, the index of its first pair in
 * fw_adjoint_rollout's d_mu and its pair count); any pointer may be NULL.  With several
 * fw_add_env_bodies calls of different structures, this is how a caller finds a body.  A
 * pile env has no listed pairs: first_pair = n_pairs = -1 (its pairs: fw_get_pile_pairs).
 * Errors: FW_ERR_ARG for env outside 0..n_envs-1. */
FW_API fw_status fw_get_env_info(fw_world *w, int env, int *first_body, int *n_bodies, int *first_pair,
                                 int *n_pairs);

/* Number of kernel launches one fw_step(n_substeps, ...) enqueues. */
FW_API int fw_launches_per_step(fw_world *w, int n_substeps);

/* Message of the last failed call on this world (never NULL). */
FW_API const char *fw_last_error(const fw_world *w);

/* ---------------------------------------------------------------- measurement */
/* L2 read bandwidth of a device, the denominator of the L2 roofline of kernels whose
 * working set stays in L2 (not on the substep path; no counterpart in the paper).
 * Allocates a device buffer of `bytes` (a multiple of 16, far below the L2 size), fills
 * it, reads it once to bring it into L2, then times `iters` full reads by SM-count x 8
 * blocks of 16-byte loads that bypass L1, and frees it.  *gbs = iters x bytes / time
 * (GB/s, 1e9 bytes).  Synchronises; runs on a stream of its own.
 * Errors: FW_ERR_ARG for bytes < 1 MiB, bytes not a multiple of 16, iters < 1 or a NULL
 * gbs; FW_ERR_CUDA if a CUDA call fails. */
FW_API fw_status fw_measure_l2_read(int device, long long bytes, int iters, float *gbs);

#ifdef __cplusplus
}
#endif
#endif /* FW_H */
