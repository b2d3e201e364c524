// fw_internal.h -- structures shared by libfw's host code and kernels.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/fw.h"

namespace fw {

constexpr int kBatch = 1024;        // Generate batch of Algorithm 1 (Sec. III-C)
constexpr int kSlots = 7;           // per patch: deepest + 6 direction extremes
constexpr int kMaxPatchesCap = 256; // upper end of the paper's 128 <= N <= 256

// device status word bits
constexpr unsigned kStatusNonFinite = 1u;
constexpr unsigned kStatusOverflow = 2u;
constexpr unsigned kStatusBounds = 4u;
constexpr unsigned kStatusTimeout = 8u;   // a bounded device wait gave up

// The solve streams an env's rows into shared memory kChunk at a time; the row region of
// an env is followed by kRowPad rows that repeat its first rows (row nr + j holds row
// j mod nr), so that every chunk of the periodic row stream is one contiguous copy.
constexpr int kChunk = 16;
constexpr int kRowPad = kChunk;

// Grid view of one asset's SDF.  Value at node (i, j, k) = val[(k*ny + j)*nx + i]; FP16
// grids store phi / h.
struct AssetDev {
    const float4 *samples;   // asset-frame sample points (x, y, z, 0)
    const float *grid;       // float32 nodes (bake output; fw_get_sdf)
    // Cell-corner copy used by every query: cell (i, j, k), i < nx - 1 fastest, holds the
    // values of its 8 corners in the order 000 100 010 110 001 101 011 111 (x fastest), so
    // one query reads 32 contiguous bytes (float32, two float4) or 16 (float16 phi / h, one
    // uint4).  Exactly one of the two is set, by the world's precision.
    const float4 *cell32;
    const uint4 *cell16;
    float lo[3];
    float h, inv_h, inv_h_lo; // inv_h + inv_h_lo = 1/h to ~1e-14 relative
    int dims[3];
    int ns;
    int nt;                  // triangles of the mesh
    const float4 *tri;       // 3 per triangle: asset-frame vertices (x, y, z, 0)
    // Narrow-band bricked storage (world option sdf_band > 0): cells grouped in bricks of
    // kBrick^3; brick[b] is the slot of a stored brick in cell32/cell16 (kBrickCells cells
    // each, x fastest inside the brick), or -1 / -2 for a brick left out because all its
    // nodes are above +band / below -band.  NULL: dense cell-corner copy.
    const int *brick;
    int bdims[3];            // bricks per axis
    float band;              // metres
    float radius;            // bounding sphere about the asset origin: every vertex and sample
    // per group of kCullGroup consecutive samples (the samples come sorted along a space-
    // filling curve): a bounding sphere (centre in the asset frame, radius rounded up); NULL
    // without samples
    const float4 *spheres;
};
constexpr int kCullGroup = 32;   // samples per bounding sphere of the query's cull (one warp's)

struct BodyProps {           // constant per body
    int type, asset;
    float invm, mass;
    float com_b[3];
    float Ib[6];             // inertia about the COM, asset frame: xx yy zz xy xz yz
    float Ib_inv[6];
    float axis[3];
    float force[3], torque[3];
    float mu;
    float pad_[3];
};

struct PairDev {
    int a, b;                // global body ids (a: sample points, b: SDF)
    int asset_a, asset_b;
    int env;
    int scratch_off;         // offset (in float4) of this pair's per-sample scratch
    float mu;                // sqrt(mu_a mu_b)
    int local_a, local_b;    // body ids within the env
    int pad_[3];
};

// The pose of one pair as a single affine map from body A's frame into body B's grid
// coordinates: u = A s + f + c for a sample s, A = R_B^T R_A / h (row-major), and the
// translation (R_B^T (p_A - p_B) - lo) / h split into an integer part c (exact) and a
// remainder f in [0, 1).  Formed in FP64 once per pair and substep, rounded once.
struct __align__(16) PairMap {
    float A[9];
    float f[3];
    int c[3];
    int pad_;
};

struct EnvDev {
    int first_body, n_bodies;
    int first_pair, n_pairs;
    int row_off;             // offset of the env's rows in the row buffer
    int row_cap;             // rows available to the env
    int movable;             // local id of the only movable body, -1 none, -2 several
    int pile;                // index of the env's pile (PileDev), -1 for an env of listed pairs
};
// Row-buffer slots (Row) an env's region spans: its rows and the kRowPad repeat rows; an env
// of several movable bodies takes two slots per row (its two-body fast rows, kPileRowF4
// float4 each, when the solve runs them).
inline long long env_row_span(const EnvDev &E) { return (E.movable == -2 ? 2LL : 1LL) * E.row_cap + kRowPad; }

// A pile env: up to kMaxPileBodies bodies whose pairs a broad phase finds at every detection
// (pile_pairs_kernel), solved colour by colour (pile_solve_kernel).  Its pairs, items,
// contacts, candidates and rows live in regions of the world's pile buffers: pairs
// [pair0, pair0 + pcap), items [item0, item0 + icap), rows [row0, row0 + rcap).
struct PileDev {
    int env, first_body, n_bodies;
    int pair0, pcap;         // pair region (global pair index into the pile pair buffers)
    int item0, icap;         // item region
    int row0, rcap;          // row region
    int stride;              // per-pair scratch stride in float4 (2 x the largest sample count)
    int pad_[2];
};
constexpr int kMaxPileBodies = 1024;
constexpr int kPilePairsPerBody = 8;    // pair capacity per body of a pile
constexpr int kPileRowsPerBody = 192;   // row (contact) capacity per body of a pile
constexpr int kPileRowF4 = 28;          // float4 per pile row (the two-body fast form of the sweeps)
constexpr int kMaxColors = 64;          // pair colours of a pile solve; the last gathers the rest

// A reduced contact on the device.  sample_patch = sample | (patch << 24).
struct __align__(16) DContact {
    float xa[3];
    float phi;
    float n[3];
    int sample_patch;
};

// One contact's constraint rows (normal, tangent 1, tangent 2), Sec. III-B.
struct __align__(16) Row {
    float n[3], t1[3], t2[3];          // directions (world)
    float ra_n[3], ra_t1[3], ra_t2[3]; // r_A x d
    float rb_n[3], rb_t1[3], rb_t2[3]; // r_B x d
    float ia_n[3], ia_t1[3], ia_t2[3]; // I_A^-1 (r_A x d)
    float ib_n[3], ib_t1[3], ib_t2[3]; // I_B^-1 (r_B x d)
    float kn, kt1, kt2, bias;          // effective masses, bias velocity
    float mu, ln, lt1, lt2;            // friction coefficient, accumulated impulses
    int a, b;                          // local body ids
    int pad_[2];
};

struct SimParams {
    const AssetDev *assets;
    const PairDev *pairs;
    const EnvDev *envs;
    const BodyProps *props;
    float *pos, *quat, *linvel, *angvel;   // state (n_bodies x 3 / 4)
    DContact *contacts;                    // n_pairs x cap_pair
    int *counts;                           // n_pairs
    float4 *scratch;                       // per pair per sample: (x, phi), (n, 0)
    Row *rows;
    unsigned *status;
    int n_pairs, n_envs, cap_pair, max_patches;
    float contact_offset, cos_patch, baumgarte, max_angvel;
    float gravity[3];
    float hs;
    int n_iters, n_vel_iters;
    int lam_cap;                           // rows whose impulses fit in shared memory (fast path)
    // detection work list: item k = (pair, batch of kBatch samples); a pair's items are
    // contiguous, pair_item0[pair] .. pair_item0[pair + 1] - 1, in batch order
    const int2 *items;
    const int *pair_item0;
    int n_items;
    float4 *cand;                          // n_items x kBatch x 2: (x_w, phi), (n_w, sample)
    int *cand_count;                       // n_items
    PairMap *maps;                         // n_pairs: each pair's map into its SDF grid
    // pile launches (pile_counts non-null): pairs, items and contacts are the pile buffers,
    // laid out in regions of pile_pcap pairs and pile_icap items per pile; pile_counts[k] =
    // (pairs, items) found for pile k, item_range[pair] = its items [x, y)
    const int2 *pile_counts;
    const int2 *item_range;
    int pile_pcap, pile_icap;
    int contact_gen;                       // 0: per sample, 1: per triangle (local minimisation)
    int multi_movable;                     // some env has several movable bodies (general sweep form)
    int sdf_bricks;                        // the assets' SDFs are held in narrow-band bricks
    int solver;                            // 0: Gauss-Seidel; 1: weighted Jacobi
    int broad_phase;                       // some env has several pairs: skip pairs far apart
    int query_threads;                     // per-sample query CTA size (128, 256, 512; 0: 256)
    int reduce_warps;                      // reduction warps per pair (2, 4, 8; 0: 4)
    int cull;                              // the query's bounding-sphere cull of sample groups
    unsigned *cull_mask;                   // per item: bit g set when its sample group g is culled
                                           // (written by map_kernel; NULL: no cull)
    int stall;                             // test hook (fw_test_stall): 1 the pile sweeps' grid
                                           // barriers wait for one block too many, 2 the
                                           // solve's row stream issues no copy
    int tri_iters;                         // descent steps per triangle
};

constexpr int kBrickLog = 3;                          // narrow-band bricks of 8^3 cells
constexpr int kBrick = 1 << kBrickLog;
constexpr int kBrickCells = kBrick * kBrick * kBrick;

// launchers (defined in the .cu files)
cudaError_t launch_bake(const float *d_tri, int n_tri, const float *d_tri_pn, const float *d_tile_box,
                        const AssetDev &g, float *d_out, int *d_flags, cudaStream_t s);
cudaError_t launch_bake_fix_sign(const float *d_tri, int n_tri, const AssetDev &g, float *d_out,
                                 const int *d_idx, int n_idx, cudaStream_t s);
cudaError_t launch_cells(const float *grid, const int dims[3], float inv_h, float4 *cell32, uint4 *cell16,
                         cudaStream_t s);   // one of cell32 / cell16 non-null
int bake_tile_size();
// narrow-band bricks: per brick 1 (stored), -1 or -2 (out of band outside / inside)
cudaError_t launch_brick_flags(const float *grid, const int dims[3], float band, const int bdims[3], int *flags,
                               cudaStream_t s);
// cell-corner copies of the stored bricks (one of cell32 / cell16 non-null)
cudaError_t launch_brick_cells(const float *grid, const int dims[3], float inv_h, const int bdims[3],
                               const int *brick_of_slot, int n_stored, float4 *cell32, uint4 *cell16, cudaStream_t s);
cudaError_t launch_query_sdf(const AssetDev &g, const float *pts, int n, float *phi, float *grad,
                             cudaStream_t s);
cudaError_t launch_query_pair(const SimParams &p, int pair, float *phi, float *nrm, cudaStream_t s, int ns);
cudaError_t prepare_detect(int max_patches);
cudaError_t launch_query(const SimParams &p, cudaStream_t s);    // narrow phase of every work item
cudaError_t launch_reduce(const SimParams &p, cudaStream_t s);   // Algorithm 1 of every pair
cudaError_t launch_detect(const SimParams &p, cudaStream_t s);   // both
// every pile's pairs, items and item ranges from the broad phase (one block per pile)
cudaError_t launch_pile_pairs(const SimParams &p, const PileDev *piles, int n_piles, PairDev *pairs, int2 *items,
                              int2 *item_range, int2 *counts, cudaStream_t s);
constexpr int kNoAllocMaxSamples = 65536;   // sample ids accepted by fw_reduce_noalloc
cudaError_t launch_reduce_noalloc(const SimParams &p, int device, const float *d_cands, int n, fw_contact *d_out,
                                  int cap, int *d_counts, cudaStream_t s);
cudaError_t launch_reduce_list(const SimParams &p, const float *d_cands, int n, DContact *out,
                               int *d_count, int *d_npatch, cudaStream_t s);
constexpr int kLamCapMax = 4096;   // fast-path impulse rows per env held in shared memory
constexpr int kMaxPairsPerEnv = 63;
constexpr int kSolveMaxWarps = 4;  // warps per solve block (one per scheduler of an SM)
// Launch shape of the solve: `groups` envs per warp (32 / groups lanes each), `warps` warps
// per block, `smem` dynamic shared memory per block.
struct SolveShape {
    int groups, warps;
    size_t smem;
};
size_t solve_smem_bytes(int lam_cap);
// Differentiable rollout (fw_diff.cu owns the layouts behind the void pointers).
struct DiffState {
    int S = 0, K = 0, row_cap = 0;
    float hs = 0.f;
    int *dyn = nullptr;               // per env: the dynamic body (global id) or -1
    void *tape_c = nullptr;           // S * n_envs * row_cap contact records (sample, pair, cell, flags)
    int *tape_n = nullptr;            // S * n_envs
    unsigned char *tape_r = nullptr;  // S * n_envs * row_cap * K decision bits
    unsigned char *tape_b = nullptr;  // S * n_envs clamp bits
    float *ck = nullptr;              // S checkpoints: pos | quat | lin | ang blocks of S * n_bodies
    float *scratch = nullptr;         // 13 * n_bodies
    void *rows = nullptr, *rbar = nullptr;   // n_envs * row_cap each
    float *upd = nullptr, *lam = nullptr, *xb = nullptr, *mass_b = nullptr, *mu_row = nullptr, *mu_b = nullptr;
};
size_t diff_tape_record_bytes();
size_t diff_row_bytes();
size_t diff_row_bar_bytes();
cudaError_t launch_diff_forward(const SimParams &p, const DiffState &d, int si, int n_bodies, bool replay,
                                cudaStream_t s);
cudaError_t launch_diff_reverse(const SimParams &p, const DiffState &d, int si, int n_bodies, cudaStream_t s);

// Allows each solve instance (1, 2, 4, 8 envs per warp) the largest dynamic shared memory
// that fits beside its static part in `optin` bytes; returns those limits in max_dyn.
cudaError_t prepare_solve(int optin, int max_dyn[4]);
// groups / warps <= 0 choose automatically: as few envs per warp as still give every
// scheduler of the device (n_sm x 4) at most about one warp.
SolveShape solve_shape(int n_envs, int lam_cap, int groups, int warps, const int max_dyn[4], int n_sm);
cudaError_t launch_solve(const SimParams &p, const SolveShape &sh, cudaStream_t s);
cudaError_t launch_normalize_quats(float *quat, int n, cudaStream_t s);
// The pile solve's tables in global memory: prepared by one block per pile
// (pile_prep_kernel), then read by the sweeps spread over the whole GPU (pile_sweep_kernel).
// Per-pair arrays and `order` are in pile regions like the pair buffers.
struct PileSolveMem {
    unsigned char *color;     // per pair: its colour in the last solve, 255 without rows
    unsigned *ab, *rr;        // per pair: a | b << 16 (+ movable bits 15, 31), rows start | count << 21
    int *order;               // the pairs with rows by colour
    int *cstart;              // per pile: kMaxColors + 1 colour starts into `order`
    int *ncol;                // per pile: colours used
    float4 *bv, *bw, *bcom;   // per body (global id): velocity | inverse mass, angular velocity |
                              // movable (1 or 0), centre of mass (world)
    float4 *binv;             // per body: the world inverse inertia's six words (xx yy zz xy | xz yz - -)
    unsigned *bar;            // the sweep kernel's grid-barrier counter
};
// The pile solve keeps per-pair tables in shared memory: a pair's rows as start | count << 21
// and pair indices as 16 bits, hence these limits on a pile's capacities.
constexpr int kPileMaxRows = 1 << 21;
constexpr int kPileMaxPairs = 65535;
size_t pile_smem_bytes(int n_bodies, int pcap);
// *max_dyn: the prep kernel's dynamic shared memory allowed; *sweep_blocks: blocks of the
// cooperative sweep kernel (all resident at once) on `device`
cudaError_t prepare_pile_solve(int optin, int device, int *max_dyn, int *sweep_blocks);
cudaError_t launch_pile_solve(const SimParams &p, const PileDev *piles, int n_piles, const int2 *counts,
                              const PileSolveMem &m, float4 *rows, size_t smem, int sweep_blocks, cudaStream_t s);
cudaError_t launch_tri_pair(const SimParams &p, int pair, float *x, float *phi, float *nrm, cudaStream_t s, int nt);
cudaError_t measure_l2_read(int device, long long bytes, int iters, float *gbs);

}  // namespace fw
