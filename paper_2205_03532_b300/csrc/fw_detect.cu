// fw_detect.cu -- SDF narrow phase and contact reduction (Sec. III-A, III-C, Algorithm 1),
// two kernels per substep.
//
// query_kernel<kTri, kStore>: one CTA of 256 threads per work item (pair, Generate batch
// of 1024 samples or faces).  Per sample (kTri false) each thread queries 4 samples --
// coalesced float4 sample loads, the 8-corner gathers of all four in flight together; per
// face (kTri true, contact_gen = 1) each thread streams the descent steps of its 4 faces
// (tri_batch).  The CTA compacts the candidates (phi < contact offset) in sample or face
// order into the item's slab of the candidate buffer: per candidate the float4 pair
// (x_w, phi), (n_w, index).  kStore selects dense or narrow-band bricked SDF storage.  In
// worlds whose envs hold several pairs, an item whose bodies' bounding spheres are too
// far apart to touch is skipped (broad phase).
//
// reduce_kernel: one CTA of kReduceWarps warps per pair runs Algorithm 1 over the pair's
// items in batch order.  It stages a batch's candidates in shared memory (read in place
// from global memory when there are more than kStage), assigns them to the existing
// patches (64-bit shared atomics pick each slot's winner), ranks the rest by depth, and
// turns them into new patches in rounds: one warp takes the kWinR deepest unassigned
// candidates and finds, with one ballot per seed and 32 members, which of them FindDeepest
// would pick as patch seeds one after another (a member is a seed unless an earlier seed's
// normal is similar enough; at most kWin per round); then every thread runs BinReduce for
// all of the round's seeds at once (each
// remaining candidate joins the first seed, in depth order, whose normal is similar), and
// AddPatch takes the new patches in seed order.  The patches and contacts are those of
// the one-patch-at-a-time loop: within a round no later seed can change an earlier
// seed's members.  Patches stay in shared memory for the whole pair; only the reduced
// contacts reach global memory, plus the data of slot winners in a per-sample scratch
// line.
//
// The same reduction code, on one warp, serves fw_reduce_noalloc, and on kReduceWarps
// warps serves fw_reduce (a caller's candidate list).
#include <atomic>
#include <mutex>

#include "fw_device.cuh"

namespace fw {

namespace {

constexpr int kQueryThreads = 256;
constexpr int kQueryPerThread = kBatch / kQueryThreads;   // 4 samples per thread
constexpr int kReduceWarps = 4;
constexpr int kStage = 256;              // candidates of a batch staged in shared memory
constexpr int kWin = 32;                 // new patches (seeds) per round at most
constexpr int kWinR = 128;               // deepest unassigned candidates examined per round
static_assert(kWinR <= kBatch, "the round's window reuses the batch's candidate list");

__constant__ float c_cos6[6] = {1.0f, 0.5f, -0.5f, -1.0f, -0.5f, 0.5f};
__constant__ float c_sin6[6] = {0.0f, 0.8660254037844386f, 0.8660254037844386f, 0.0f,
                                -0.8660254037844386f, -0.8660254037844386f};

// Patch state of one pair in shared memory.  NP = max_patches + kWin: the patches kept,
// then the kWin slots of a round's new patches.  Of a patch's tangent basis only t1 is
// stored; t2 = n x t1 is formed again where needed (patch_t2, explicitly rounded, so it is
// the same vector at every use).
struct PatchSm {
    float4 *pn4;                  // NP patch normals (x, y, z, 0)
    unsigned *kord;               // kBatch: depth keys ord(phi) of the unassigned candidates
                                  // (in cl's order), then the depth order itself
    unsigned long long *keys;     // kSlots x NP
    float *pa, *pt1;              // 3 x NP each, component-major: anchor, tangent t1
    short *cst;                   // kBatch: -1 unassigned, -3 consumed, >= 0 existing patch,
                                  // -4 - t joining the round's new patch t
    short *cl;                    // kBatch: the unassigned candidates of the batch
    int *npat;                    // patches kept
    int *nun;                     // unassigned candidates of the batch
    int *nseed;                   // new patches of the round
    int *win;                     // kWin: the round's seeds (candidate ids, seed order)
    short *wcand;                 // kWinR: the round's window (candidate ids, depth order); it
                                  // reuses cl, dead once the depth order is built
};

__host__ __device__ inline size_t patch_smem_bytes(int NP) {
    size_t b = (size_t)NP * 16 + (size_t)kBatch * 4 + (size_t)kSlots * NP * 8 + (size_t)6 * NP * 4;
    b = (b + 7) & ~(size_t)7;
    b += (size_t)kBatch * 4;                  // cst, cl
    b += 16 + (size_t)kWin * 4;               // npat, nun, nseed (+ pad), win
    return (b + 15) & ~(size_t)15;
}

__device__ __forceinline__ PatchSm carve_patch(unsigned char *base, int NP) {
    PatchSm s;
    s.pn4 = reinterpret_cast<float4 *>(base);                      // 16-byte aligned
    s.kord = reinterpret_cast<unsigned *>(s.pn4 + NP);             // 16-byte aligned
    s.keys = reinterpret_cast<unsigned long long *>(s.kord + kBatch);
    s.pa = reinterpret_cast<float *>(s.keys + kSlots * NP);
    s.pt1 = s.pa + 3 * NP;
    size_t off = (size_t)NP * 16 + (size_t)kBatch * 4 + (size_t)kSlots * NP * 8 + (size_t)6 * NP * 4;
    off = (off + 7) & ~(size_t)7;
    s.cst = reinterpret_cast<short *>(base + off);
    s.cl = s.cst + kBatch;
    off += (size_t)kBatch * 4;
    int *ip = reinterpret_cast<int *>(base + off);
    s.npat = ip; s.nun = ip + 1; s.nseed = ip + 2;
    s.win = ip + 4;
    s.wcand = s.cl;
    return s;
}

// candidate c of a batch: cd[2c] = (x_w, phi), cd[2c + 1] = (n_w, sample as int bits)
__device__ __forceinline__ V3 cpos(const float4 *cd, int c) { const float4 a = cd[2 * c]; return v3(a.x, a.y, a.z); }
__device__ __forceinline__ float cphi(const float4 *cd, int c) { return cd[2 * c].w; }
__device__ __forceinline__ V3 cnrm(const float4 *cd, int c) { const float4 b = cd[2 * c + 1]; return v3(b.x, b.y, b.z); }
__device__ __forceinline__ int cidx(const float4 *cd, int c) { return __float_as_int(cd[2 * c + 1].w); }

// normal similarity n . m, rounded the same way wherever a decision compares it (and
// symmetric: ndot(a, b) == ndot(b, a) bit for bit)
__device__ __forceinline__ float ndot(V3 a, V3 b) { return __fmaf_rn(a.z, b.z, __fmaf_rn(a.y, b.y, a.x * b.x)); }
__device__ __forceinline__ float ndot(V3 a, float4 b) { return ndot(a, v3(b.x, b.y, b.z)); }

// second tangent of a patch: n x t1, each component rounded in one fixed way
__device__ __forceinline__ V3 patch_t2(V3 n, V3 t1) {
    return v3(__fmaf_rn(n.y, t1.z, -__fmul_rn(n.z, t1.y)), __fmaf_rn(n.z, t1.x, -__fmul_rn(n.x, t1.z)),
              __fmaf_rn(n.x, t1.y, -__fmul_rn(n.y, t1.x)));
}

// Per-pair transform.
struct PairXf {
    M3 RA, RB;
    V3 pA, pB;
};

__device__ __forceinline__ void load_pose(const SimParams &p, int body, M3 &R, V3 &t) {
    const float4 q = make_float4(p.quat[4 * body], p.quat[4 * body + 1], p.quat[4 * body + 2], p.quat[4 * body + 3]);
    R = quat_to_mat(q);
    t = ld3(p.pos + 3 * body);
}

// Column i of the rotation of q = (x, y, z, w) (row i of its transpose), in FP64.
__device__ __forceinline__ void rot_col(const float *q, int i, double r[3]) {
    const double x = q[0], y = q[1], z = q[2], w = q[3];
    if (i == 0) { r[0] = 1.0 - 2.0 * (y * y + z * z); r[1] = 2.0 * (x * y + z * w); r[2] = 2.0 * (x * z - y * w); }
    else if (i == 1) { r[0] = 2.0 * (x * y - z * w); r[1] = 1.0 - 2.0 * (x * x + z * z); r[2] = 2.0 * (y * z + x * w); }
    else { r[0] = 2.0 * (x * z + y * w); r[1] = 2.0 * (y * z - x * w); r[2] = 1.0 - 2.0 * (x * x + y * y); }
}

// The map of pair P into body B's grid (PairMap), by one thread in FP64 from the float32
// quaternions and positions; 1/h is the stored float pair inv_h + inv_h_lo (1/h to ~1e-14).
// Formed once per pair and substep (map_kernel) and the same way, by this one function, for
// the per-pair test hook.  A point whose translation is not finite gets a cell far outside.
__device__ __noinline__ void pair_map(const SimParams &p, const PairDev &P, const AssetDev &gb, PairMap &M) {
    const float *qa = p.quat + 4 * P.a, *qb = p.quat + 4 * P.b;
    const double inv_h = (double)gb.inv_h + (double)gb.inv_h_lo;
    const double d[3] = {(double)p.pos[3 * P.a] - p.pos[3 * P.b], (double)p.pos[3 * P.a + 1] - p.pos[3 * P.b + 1],
                         (double)p.pos[3 * P.a + 2] - p.pos[3 * P.b + 2]};
    double ra[3][3];
    for (int j = 0; j < 3; ++j) rot_col(qa, j, ra[j]);
    for (int i = 0; i < 3; ++i) {
        double rb[3];
        rot_col(qb, i, rb);
        for (int j = 0; j < 3; ++j)
            M.A[3 * i + j] = (float)((rb[0] * ra[j][0] + rb[1] * ra[j][1] + rb[2] * ra[j][2]) * inv_h);
        const double u = ((rb[0] * d[0] + rb[1] * d[1] + rb[2] * d[2]) - (double)gb.lo[i]) * inv_h;
        const double fl = floor(u);
        const bool finite = fl == fl && fabs(fl) < 1.0e6;
        M.c[i] = finite ? (int)fl : -(1 << 28);
        M.f[i] = finite ? (float)(u - fl) : 0.0f;
    }
    M.pad_ = 0;
}

// Whether no sample of a group can be a candidate, from its bounding sphere sp (centre in
// the frame of the pair's point body, radius): the sphere lies outside the grid box of the
// SDF body gb on some axis (a sample outside the grid is no candidate), or the SDF at its
// centre exceeds the cutoff by more than the interpolated field can change over the radius
// (at most sqrt(3) per unit length for a distance field; 2.5 covers FP16 rounding), plus a
// voxel.  Dense storage (a narrow band's clamped values do not bound the field).
template <bool kHalf>
__device__ __forceinline__ bool group_culled_as(const PairMap &M, const AssetDev &gb, float4 sp, float cutoff) {
    const float u[3] = {__fmaf_rn(M.A[2], sp.z, __fmaf_rn(M.A[1], sp.y, __fmaf_rn(M.A[0], sp.x, M.f[0]))),
                        __fmaf_rn(M.A[5], sp.z, __fmaf_rn(M.A[4], sp.y, __fmaf_rn(M.A[3], sp.x, M.f[1]))),
                        __fmaf_rn(M.A[8], sp.z, __fmaf_rn(M.A[7], sp.y, __fmaf_rn(M.A[6], sp.x, M.f[2])))};
    const float ru = sp.w * gb.inv_h * 1.0001f + 1e-3f;   // the radius in voxels, with a margin for the map's rounding
    for (int a = 0; a < 3; ++a) {
        const float g = u[a] + (float)M.c[a];             // the centre's grid coordinate
        if (g + ru < 0.0f || g - ru > (float)(gb.dims[a] - 1)) return true;
    }
    int ci, cj, ck;
    float fx, fy, fz;
    const bool okx = cell_of(u[0], M.c[0], gb.dims[0], ci, fx);
    const bool oky = cell_of(u[1], M.c[1], gb.dims[1], cj, fy);
    const bool okz = cell_of(u[2], M.c[2], gb.dims[2], ck, fz);
    const CellCorners c = sdf_cell_corners<kHalf, kStoreDense>(gb, ci, cj, ck);
    const float phi = cell_value<kHalf>(gb, c, fx, fy, fz);
    return okx && oky && okz && phi - 2.5f * sp.w > cutoff + gb.h;
}
__device__ __forceinline__ bool group_culled(const PairMap &M, const AssetDev &gb, float4 sp, float cutoff) {
    return gb.cell16 ? group_culled_as<true>(M, gb, sp, cutoff) : group_culled_as<false>(M, gb, sp, cutoff);
}

// Every pair's map for the coming query (one thread per pair).
__global__ void map_kernel(SimParams p) {
    const int pi = blockIdx.x * blockDim.x + threadIdx.x;
    if (pi >= p.n_pairs) return;
    if (p.pile_counts && pi % p.pile_pcap >= p.pile_counts[pi / p.pile_pcap].x) return;
    const PairDev P = p.pairs[pi];
    PairMap M;
    pair_map(p, P, p.assets[P.asset_b], M);
    p.maps[pi] = M;
}

// The maps as map_kernel forms them, and the cull masks of the pairs' items
// (fw_set_query_cull; dense storage): a block takes kCullPairs pairs; its first warp forms
// their maps, a lane per pair (an FP64 warp instruction occupies the FP64 pipe for the whole
// warp however few lanes are active, so the maps are formed by as few warps as they are in
// map_kernel), then warp w tests pair w's groups: bit g of an item's mask, from lane g, is set
// when the item's samples 32 g .. 32 g + 31 can be no candidate (group_culled).
constexpr int kCullPairs = 16;
__global__ void __launch_bounds__(32 * kCullPairs, 2) map_cull_kernel(SimParams p) {
    __shared__ PairMap maps[kCullPairs];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, p0 = blockIdx.x * kCullPairs;
    if (warp == 0 && lane < kCullPairs) {
        const int pi = p0 + lane;
        if (pi < p.n_pairs && !(p.pile_counts && pi % p.pile_pcap >= p.pile_counts[pi / p.pile_pcap].x)) {
            const PairDev P = p.pairs[pi];
            PairMap M;
            pair_map(p, P, p.assets[P.asset_b], M);
            p.maps[pi] = M;
            maps[lane] = M;
        }
    }
    __syncthreads();
    const int pi = p0 + warp;
    if (pi >= p.n_pairs) return;   // the same on every lane of the warp
    if (p.pile_counts && pi % p.pile_pcap >= p.pile_counts[pi / p.pile_pcap].x) return;   // past a pile's pairs
    const PairDev P = p.pairs[pi];
    const AssetDev ga = p.assets[P.asset_a], gb = p.assets[P.asset_b];
    if (p.broad_phase) {   // the query skips the pair's items (query_kernel): no mask is read
        const V3 dp = ld3(p.pos + 3 * P.a) - ld3(p.pos + 3 * P.b);
        const float lim = ga.radius + gb.radius + p.contact_offset + 2.0f * gb.h;
        if (dot(dp, dp) > lim * lim) return;
    }
    // the pair's items: batch it - i0 of its samples is item it
    const int i0 = p.item_range ? p.item_range[pi].x : p.pair_item0[pi];
    const int i1 = p.item_range ? p.item_range[pi].y : p.pair_item0[pi + 1];
    if (ga.spheres == nullptr || gb.brick != nullptr) {
        for (int it = i0 + lane; it < i1; it += 32) p.cull_mask[it] = 0u;
        return;
    }
    const PairMap M = maps[warp];
    static_assert(kBatch / kCullGroup == 32, "one cull-mask bit per lane");
    constexpr int kU = 4;   // items tested at once: their loads in flight together
    for (int b0 = i0; b0 < i1; b0 += kU) {
        float4 sp[kU];
        bool has[kU];
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            const int g = (b0 + k - i0) * (kBatch / kCullGroup) + lane;
            has[k] = b0 + k < i1 && g * kCullGroup < ga.ns;
            sp[k] = has[k] ? __ldg(&ga.spheres[g]) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        bool culled[kU];
#pragma unroll
        for (int k = 0; k < kU; ++k) culled[k] = has[k] && group_culled(M, gb, sp[k], p.contact_offset);
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            const unsigned m = __ballot_sync(0xffffffffu, culled[k]);
            if (lane == 0 && b0 + k < i1) p.cull_mask[b0 + k] = m;
        }
    }
}

// The narrow phase of one sample through the pair's map, in the grid's storage precision.
// A candidate needs phi below the cutoff first: the gradient, the world normal and the world
// point are formed only for such samples (whole warps of samples far from the SDF body
// skip them; the values are those the full lookup would give).
template <int kStore, bool kHalf>
__device__ __forceinline__ bool query_sample_as(const PairMap &M, const PairXf &X, const AssetDev &gb, float4 s,
                                                float cutoff, V3 &xw, V3 &nw, float &phi) {
    const float ux = __fmaf_rn(M.A[2], s.z, __fmaf_rn(M.A[1], s.y, __fmaf_rn(M.A[0], s.x, M.f[0])));
    const float uy = __fmaf_rn(M.A[5], s.z, __fmaf_rn(M.A[4], s.y, __fmaf_rn(M.A[3], s.x, M.f[1])));
    const float uz = __fmaf_rn(M.A[8], s.z, __fmaf_rn(M.A[7], s.y, __fmaf_rn(M.A[6], s.x, M.f[2])));
    int ci, cj, ck;
    float fx, fy, fz;
    const bool okx = cell_of(ux, M.c[0], gb.dims[0], ci, fx);
    const bool oky = cell_of(uy, M.c[1], gb.dims[1], cj, fy);
    const bool okz = cell_of(uz, M.c[2], gb.dims[2], ck, fz);
    const CellCorners c = sdf_cell_corners<kHalf, kStore>(gb, ci, cj, ck);
    phi = cell_value<kHalf>(gb, c, fx, fy, fz);
    if (!(okx && oky && okz && phi < cutoff)) return false;
    const V3 g = cell_gradient<kHalf>(gb, c, fx, fy, fz);
    const float gg = dot(g, g);
    const V3 nb = rsqrtf(fmaxf(gg, 1e-30f)) * g;   // unit to a few ulp; the decisions on it have margins
    nw = mul(X.RB, nb);
    xw = mul(X.RA, v3(s.x, s.y, s.z)) + X.pA;
    return gg >= 1e-24f;
}

// The narrow phase of one sample through the pair's map: true for a candidate (inside the
// grid, phi below the cutoff, |grad| >= 1e-12), with its signed distance, world normal
// (R_B g / |g|, float32) and world point (R_A s + p_A).
template <int kStore = kStoreAny>
__device__ __forceinline__ bool query_sample(const PairMap &M, const PairXf &X, const AssetDev &gb, float4 s,
                                             float cutoff, V3 &xw, V3 &nw, float &phi) {
    return gb.cell16 ? query_sample_as<kStore, true>(M, X, gb, s, cutoff, xw, nw, phi)
                     : query_sample_as<kStore, false>(M, X, gb, s, cutoff, xw, nw, phi);
}

// Closest point of the triangle (a, b, c) to p: p's Voronoi region among the vertices,
// the edges and the face, then the point of that feature (the standard construction of
// real-time collision detection; Ericson, Sec. 5.1.5).
__device__ V3 tri_closest(V3 p, V3 a, V3 b, V3 c) {
    const V3 ab = b - a, ac = c - a, ap = p - a;
    const float d1 = dot(ab, ap), d2 = dot(ac, ap);
    if (d1 <= 0.0f && d2 <= 0.0f) return a;
    const V3 bp = p - b;
    const float d3 = dot(ab, bp), d4 = dot(ac, bp);
    if (d3 >= 0.0f && d4 <= d3) return b;
    const V3 cp = p - c;
    const float d5 = dot(ab, cp), d6 = dot(ac, cp);
    if (d6 >= 0.0f && d5 <= d6) return c;
    const float vc = d1 * d4 - d3 * d2;                       // weight of c
    if (vc <= 0.0f && d1 >= 0.0f && d3 <= 0.0f) return a + (d1 / (d1 - d3)) * ab;
    const float vb = d5 * d2 - d1 * d6;                       // weight of b
    if (vb <= 0.0f && d2 >= 0.0f && d6 <= 0.0f) return a + (d2 / (d2 - d6)) * ac;
    const float va = d3 * d6 - d5 * d4;                       // weight of a
    if (va <= 0.0f && d4 - d3 >= 0.0f && d5 - d6 >= 0.0f)
        return b + ((d4 - d3) / ((d4 - d3) + (d5 - d6))) * (c - b);
    const float den = 1.0f / (va + vb + vc);
    return a + (vb * den) * ab + (vc * den) * ac;
}

// Per-triangle Generate (Sec. III-A): the minimiser of the SDF over the face (a, b, c),
// all in the SDF's frame, by projected gradient descent with adaptive steps -- start at
// the centroid with step length half the longest edge; each step moves against the
// gradient's in-plane part, projects onto the face and is accepted if phi decreases (step
// x 1.5), else rejected (step x 0.5); it ends after `iters` steps or when the in-plane
// gradient falls below 1e-9.  False when the centroid lies outside the grid; trial points
// outside the grid are rejected.
template <int kStore = kStoreAny>
__device__ bool tri_minimise(const AssetDev &gb, V3 a, V3 b, V3 c, int iters, V3 &x, float &phi, V3 &g) {
    const V3 e1 = b - a, e2 = c - a, e3 = c - b;
    V3 nt = cross(e1, e2);
    const float nn = dot(nt, nt);
    nt = nn > 0.0f ? rsqrtf(nn) * nt : v3(0.0f, 0.0f, 0.0f);
    x = (1.0f / 3.0f) * ((a + b) + c);
    if (!sdf_lookup_any<kStore>(gb, x, phi, g)) return false;
    float s = 0.5f * sqrtf(fmaxf(dot(e1, e1), fmaxf(dot(e2, e2), dot(e3, e3))));
    for (int it = 0; it < iters; ++it) {
        const V3 d = g - dot(g, nt) * nt;
        const float dd = dot(d, d);
        if (!(dd > 1e-18f)) break;
        const V3 xt = tri_closest(x - (s * rsqrtf(dd)) * d, a, b, c);
        float pt;
        V3 gt;
        if (sdf_lookup_any<kStore>(gb, xt, pt, gt) && pt < phi) {
            x = xt; phi = pt; g = gt;
            s *= 1.5f;
        } else {
            s *= 0.5f;
        }
    }
    return true;
}

// Triangle t of body a's mesh, minimised against body b's SDF: world point on the face,
// world normal, phi.  False when there is no candidate point (centroid outside the grid,
// vanishing gradient).
template <int kStore = kStoreAny>
__device__ __forceinline__ bool tri_sample(const PairXf &X, const AssetDev &ga, const AssetDev &gb, int t, int iters,
                                           V3 &xw, V3 &nw, float &phi) {
    V3 v[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float4 s = __ldg(&ga.tri[3 * t + k]);
        v[k] = mul_t(X.RB, mul(X.RA, v3(s.x, s.y, s.z)) + X.pA - X.pB);
    }
    V3 x, g;
    const bool in = tri_minimise<kStore>(gb, v[0], v[1], v[2], iters, x, phi, g);
    const float gg = dot(g, g);
    nw = mul(X.RB, rsqrtf(fmaxf(gg, 1e-30f)) * g);
    xw = mul(X.RB, x) + X.pB;
    return in && (gg >= 1e-24f);
}

// Per-triangle Generate of one work item, one descent step per loop trip.  A thread takes
// its faces u * kQueryThreads + tid (u = 0 .. kQueryPerThread - 1) one after another and
// starts the next face as soon as one ends, so a warp's lanes stay busy while their faces
// need different numbers of steps; the steps of a face are exactly those of tri_minimise
// (centroid lookup, then up to `iters` projected steps while the in-plane gradient is
// above 1e-9), and every trip makes at most one SDF lookup from one place in the code.
// The pose X is read from shared memory.  Face u's candidate goes to
// res[2 (u kQueryThreads + tid)] = (x_w, phi), res[... + 1] = (n_w, 0); bit u of the
// result is set when it is one.
template <int kStore>
__device__ unsigned tri_batch(const PairXf &X, const AssetDev &ga, const AssetDev &gb, int base, int tid, int iters,
                              float cutoff, float4 *res) {
    unsigned okb = 0;
    int u = 0, it = 0;
    bool start = true;
    V3 a = v3(0.f, 0.f, 0.f), b = a, c = a, nt = a, x = a, g = a;
    float phi = 0.0f, s = 0.0f;
    while (u < kQueryPerThread) {
        const int i = base + u * kQueryThreads + tid;
        V3 q;
        bool look = true;
        if (start) {
            const int t = i < ga.nt ? i : ga.nt - 1;
            V3 v[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float4 w4 = __ldg(&ga.tri[3 * t + k]);
                v[k] = mul_t(X.RB, mul(X.RA, v3(w4.x, w4.y, w4.z)) + X.pA - X.pB);
            }
            a = v[0]; b = v[1]; c = v[2];
            const V3 e1 = b - a, e2 = c - a, e3 = c - b;
            nt = cross(e1, e2);
            const float nn = dot(nt, nt);
            nt = nn > 0.0f ? rsqrtf(nn) * nt : v3(0.0f, 0.0f, 0.0f);
            q = (1.0f / 3.0f) * ((a + b) + c);
            s = 0.5f * sqrtf(fmaxf(dot(e1, e1), fmaxf(dot(e2, e2), dot(e3, e3))));
        } else {
            const V3 d = g - dot(g, nt) * nt;
            const float dd = dot(d, d);
            look = it < iters && dd > 1e-18f;
            q = look ? tri_closest(x - (s * rsqrtf(dd)) * d, a, b, c) : x;
        }
        float pt = 0.0f;
        V3 gt = v3(0.0f, 0.0f, 0.0f);
        bool in = false;
        if (look) in = sdf_lookup_any<kStore>(gb, q, pt, gt);
        bool done = false, cand = false;
        if (start) {
            x = q; phi = pt; g = gt; it = 0;
            start = false;
            done = !in;                       // centroid outside the grid: no candidate
        } else if (look) {
            if (in && pt < phi) {
                x = q; phi = pt; g = gt;
                s *= 1.5f;
            } else {
                s *= 0.5f;
            }
            ++it;
        } else {
            done = true;
            cand = true;
        }
        if (done) {
            const float gg = dot(g, g);
            cand = cand && gg >= 1e-24f && phi < cutoff && i < ga.nt;
            if (cand) {
                const V3 nw = mul(X.RB, rsqrtf(fmaxf(gg, 1e-30f)) * g);
                const V3 xw = mul(X.RB, x) + X.pB;
                const int o = 2 * (u * kQueryThreads + tid);
                res[o] = make_float4(xw.x, xw.y, xw.z, phi);
                res[o + 1] = make_float4(nw.x, nw.y, nw.z, 0.0f);
                okb |= 1u << u;
            }
            ++u;
            start = true;
        }
    }
    return okb;
}

__device__ __forceinline__ unsigned long long slot_key(float score, int sample) {
    return ((unsigned long long)ord_f32(score) << 32) | (unsigned)(0xFFFFFFFFu - (unsigned)sample);
}
__device__ __forceinline__ int key_sample(unsigned long long k) {
    return (int)(0xFFFFFFFFu - (unsigned)(k & 0xFFFFFFFFull));
}

// score of candidate (x, phi) for slot s of the patch with anchor a and basis t1, t2
__device__ __forceinline__ float slot_score(int s, V3 x, float phi, V3 a, V3 t1, V3 t2) {
    if (s == 0) return -phi;
    const V3 d = x - a;
    const float p1 = dot(d, t1), p2 = dot(d, t2);
    return __fmaf_rn(c_cos6[s - 1], p1, c_sin6[s - 1] * p2);
}

__device__ __forceinline__ V3 pvec(const float *base, int NP, int j) {
    return v3(base[j], base[NP + j], base[2 * NP + j]);
}
__device__ __forceinline__ void set_pvec(float *base, int NP, int j, V3 v) {
    base[j] = v.x; base[NP + j] = v.y; base[2 * NP + j] = v.z;
}

__device__ __forceinline__ void scratch_put(float4 *scr, int sample, V3 x, float phi, V3 n) {
    scr[2 * sample] = make_float4(x.x, x.y, x.z, phi);
    scr[2 * sample + 1] = make_float4(n.x, n.y, n.z, 0.0f);
}

// M = -phi_deepest + sqrt(area of the polygon through the distinct direction-slot
// points, in slot order, in the patch plane).  Reads winners' data from scratch.
__device__ float patch_measure(const PatchSm &S, int NP, int j, const float4 *scr) {
    const int deep = key_sample(S.keys[j]);
    const float phid = scr[2 * deep].w;
    const V3 a = pvec(S.pa, NP, j), t1 = pvec(S.pt1, NP, j);
    const V3 t2 = patch_t2(v3(S.pn4[j].x, S.pn4[j].y, S.pn4[j].z), t1);
    float xs[6], ys[6];
    int seen[6], n = 0;
    for (int s = 1; s < kSlots; ++s) {
        const int id = key_sample(S.keys[s * NP + j]);
        bool dup = false;
        for (int t = 0; t < n; ++t) dup |= (seen[t] == id);
        if (dup) continue;
        const float4 q = scr[2 * id];
        const V3 d = v3(q.x, q.y, q.z) - a;
        xs[n] = dot(d, t1);
        ys[n] = dot(d, t2);
        seen[n++] = id;
    }
    float area2 = 0.0f;
    for (int i = 0; i < n; ++i) {
        const int k = (i + 1 == n) ? 0 : i + 1;
        area2 += xs[i] * ys[k] - xs[k] * ys[i];
    }
    return -phid + sqrtf(0.5f * fabsf(area2));
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = (w > v) ? w : v;
    }
    return v;
}

// Barrier of a reduction block of kW warps (kW = 1: the warp alone).
template <int kW>
__device__ __forceinline__ void bsync() {
    if (kW == 1) __syncwarp();
    else __syncthreads();
}

template <int kW>
__device__ __forceinline__ void init_patches(const PatchSm &S, int NP) {
    for (int i = threadIdx.x; i < kSlots * NP; i += 32 * kW) S.keys[i] = 0ull;
    if (threadIdx.x == 0) { *S.npat = 0; *S.nun = 0; }
    bsync<kW>();
}

// Position of the i-th unassigned candidate in the depth order of the batch (phi
// ascending, ties to the lower candidate): kord[0..m) holds ord(phi) of the m unassigned
// candidates, cl[0..m) the candidates themselves, in no particular order.
__device__ __forceinline__ int depth_rank(const unsigned *kord, const short *cl, int m, int i) {
    const unsigned ki = kord[i];
    const uint4 *k4 = reinterpret_cast<const uint4 *>(kord);
    int lt = 0, eq = 0;
#pragma unroll 4
    for (int j = 0; j < (m >> 2); ++j) {
        const uint4 q = k4[j];
        lt += (q.x < ki) + (q.y < ki) + (q.z < ki) + (q.w < ki);
        eq += (q.x == ki) + (q.y == ki) + (q.z == ki) + (q.w == ki);
    }
    for (int j = m & ~3; j < m; ++j) {
        lt += kord[j] < ki;
        eq += kord[j] == ki;
    }
    if (eq > 1) {   // equal depths (rare): the lower candidate comes first
        const int ci = cl[i];
        for (int j = 0; j < m; ++j) lt += (kord[j] == ki) && (cl[j] < ci);
    }
    return lt;
}

// The same depth order by sorting: the m pairs (kord[i], cl[i]) are sorted in place,
// ascending by depth then candidate (a bitonic network over the next power of two, padded
// with keys after every real one), so that cl[r] is the candidate of depth rank r.  The keys
// are distinct (one per candidate), so the order is the one depth_rank gives.  m <= kBatch;
// executed by all 32 * kW threads, ends with a block barrier.
constexpr int kRankSort = 128;   // above this many unassigned candidates, sort instead of count
template <int kW>
__device__ void depth_sort(unsigned *kord, short *cl, int m) {
    constexpr int NT = 32 * kW;
    const int tid = threadIdx.x;
    int P = 1;
    while (P < m) P <<= 1;
    for (int i = m + tid; i < P; i += NT) {   // pads: above any finite depth and any candidate
        kord[i] = 0xFFFFFFFFu;
        cl[i] = (short)0x7FFF;
    }
    bsync<kW>();
    for (int k = 2; k <= P; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = tid; t < (P >> 1); t += NT) {
                const int i = 2 * t - (t & (j - 1)), l = i + j;   // the pair (i, i + j), i's bit j clear
                const unsigned ka = kord[i], kb = kord[l];
                const short ca = cl[i], cb = cl[l];
                const bool gt = ka > kb || (ka == kb && ca > cb);
                if (gt == ((i & k) == 0)) {   // out of this block's direction: swap
                    kord[i] = kb; kord[l] = ka;
                    cl[i] = cb; cl[l] = ca;
                }
            }
            bsync<kW>();
        }
}

__device__ __forceinline__ void copy_patch(const PatchSm &S, int NP, int from, int to) {
    S.pn4[to] = S.pn4[from];
    for (int k = 0; k < 3; ++k) {
        S.pa[k * NP + to] = S.pa[k * NP + from];
        S.pt1[k * NP + to] = S.pt1[k * NP + from];
    }
    for (int k = 0; k < kSlots; ++k) S.keys[k * NP + to] = S.keys[k * NP + from];
}

// AddPatch for the ns new patches of a round (slots T0 .. T0 + ns - 1, seed order): append
// below capacity, else replace the most similar kept patch if the new one measures
// higher, else drop it.  Executed by one warp.
__device__ void add_patches(const PatchSm &S, int NP, int T0, int ns, int max_patches, const float4 *scr) {
    const int lane = threadIdx.x & 31;
    int npat = *S.npat;
    const int fit = min(ns, max(0, max_patches - npat));
    if (lane < fit) copy_patch(S, NP, T0 + lane, npat + lane);
    npat += fit;
    for (int t = fit; t < ns; ++t) {
        const int T = T0 + t;
        const V3 nb = v3(S.pn4[T].x, S.pn4[T].y, S.pn4[T].z);
        unsigned long long bk = 0ull;
        for (int j = lane; j < npat; j += 32) {
            const unsigned long long k = ((unsigned long long)ord_f32(ndot(nb, S.pn4[j])) << 32) |
                                         (unsigned)(0xFFFFFFFFu - (unsigned)j);
            bk = (k > bk) ? k : bk;
        }
        bk = warp_max_u64(bk);
        const int ks = key_sample(bk);
        if (lane == 0 && patch_measure(S, NP, T, scr) > patch_measure(S, NP, ks, scr)) copy_patch(S, NP, T, ks);
        __syncwarp();
    }
    if (lane == 0) *S.npat = npat;
    __syncwarp();
}

// One round's seeds, by one warp.  The window is the first kWinR unassigned entries of the
// depth order from position pos on (lane l holds members l, l + 32, l + 64, l + 96).  The
// seeds are the members FindDeepest would pick one after another: the first remaining
// member is a seed, and every later member whose normal is similar enough to it
// (n . n_seed >= cos_patch) is covered and can no longer be one; at most kWin seeds per
// round, the window's uncovered rest staying for the next round.  Each seed costs one
// broadcast of its normal and one ballot per 32 members.  Writes the seeds' patch frames
// into slots T0.., their candidates into S.win and their count into *S.nseed; returns the
// position from which the next round scans (entries consumed meanwhile are skipped).
__device__ int next_seeds(const PatchSm &S, int NP, int T0, const float4 *cd, const int *order, int m, int pos,
                          float cos_patch) {
    constexpr int kQ = kWinR / 32;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    int k = 0;
    const int start = pos;
    while (k < kWinR && pos < m) {
        const int i = pos + lane;
        const int c = i < m ? order[i] : -1;
        const bool un = c >= 0 && S.cst[c] == -1;
        const unsigned b = __ballot_sync(0xffffffffu, un);
        const int nb = __popc(b), take = min(nb, kWinR - k);
        const int r = __popc(b & lt);
        if (un && r < take) S.wcand[k + r] = (short)c;
        const unsigned last = __ballot_sync(0xffffffffu, un && r == take - 1);
        pos = (take == nb) ? pos + 32 : pos + __ffs(last);
        k += take;
    }
    __syncwarp();
    V3 n[kQ];
    unsigned rem[kQ];
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
        const int idx = 32 * q + lane;
        const bool v = idx < k;
        n[q] = v ? cnrm(cd, S.wcand[idx]) : v3(0.0f, 0.0f, 0.0f);
        rem[q] = __ballot_sync(0xffffffffu, v);
    }
    int ns = 0;
    while (ns < kWin) {
        int q0 = kQ;   // first word with a remaining member (the same on every lane)
#pragma unroll
        for (int q = kQ - 1; q >= 0; --q) q0 = rem[q] ? q : q0;
        if (q0 == kQ) break;
        int l = 0;
        V3 nq = n[0];
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            if (q == q0) { l = __ffs(rem[q]) - 1; nq = n[q]; }
        }
        const V3 sd = v3(__shfl_sync(0xffffffffu, nq.x, l), __shfl_sync(0xffffffffu, nq.y, l),
                         __shfl_sync(0xffffffffu, nq.z, l));
        const int i = 32 * q0 + l;   // the seed's window index
        if (lane == 0) S.win[ns] = S.wcand[i];
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            const bool later = 32 * q + lane > i;
            const unsigned cov = __ballot_sync(0xffffffffu, later && ndot(n[q], sd) >= cos_patch);
            rem[q] &= ~cov;
        }
#pragma unroll
        for (int q = 0; q < kQ; ++q)
            if (q == q0) rem[q] &= ~(1u << l);
        ++ns;
    }
    __syncwarp();   // S.win written
    if (lane < ns) {
        const int c = S.win[lane], T = T0 + lane;
        const V3 nn = cnrm(cd, c);
        V3 t1, t2;
        tangent_basis(nn, t1, t2);
        S.pn4[T] = make_float4(nn.x, nn.y, nn.z, 0.0f);
        set_pvec(S.pa, NP, T, cpos(cd, c));
        set_pvec(S.pt1, NP, T, t1);
        for (int q = 0; q < kSlots; ++q) S.keys[q * NP + T] = 0ull;
    }
    if (lane == 0) *S.nseed = ns;
    // every window member is now a seed or covered by one (BinReduce consumes them all): the
    // next round scans on from the window's end; otherwise (kWin seeds reached) from its start
    unsigned left = 0u;
#pragma unroll
    for (int q = 0; q < kQ; ++q) left |= rem[q];
    return left ? start : pos;
}

// Algorithm 1 for one batch: nc candidates in sample order at cd (shared or global
// memory); patches persist in S.  Executed by all 32 * kW threads of the block.
template <int kW>
__device__ void reduce_batch(const PatchSm &S, int NP, const float4 *cd, int nc, int max_patches, float cos_patch,
                             float4 *scr) {
    constexpr int NT = 32 * kW;
    constexpr int kPer = kBatch / NT;
    const int tid = threadIdx.x;
    const int np0 = *S.npat;
    const int T0 = NP - kWin;
    // ---- Assign: join the most similar existing patch if similar enough
    const int lane = tid & 31;
    for (int c0 = 0; c0 < nc; c0 += NT) {   // same trip count on every lane (ballot below)
        const int c = c0 + tid;
        int best = -1;
        float bd = -3.0f;
        if (c < nc) {
            const V3 n = cnrm(cd, c);
#pragma unroll 4
            for (int j = 0; j < np0; ++j) {
                const float d = ndot(n, S.pn4[j]);
                if (d > bd) { bd = d; best = j; }
            }
        }
        // the warp's unassigned candidates take consecutive list entries
        const bool un = c < nc && !(best >= 0 && bd >= cos_patch);
        const unsigned um = __ballot_sync(0xffffffffu, un);
        int i0 = 0;
        if (lane == 0 && um) i0 = atomicAdd(S.nun, __popc(um));
        i0 = __shfl_sync(0xffffffffu, i0, 0);
        if (c >= nc) continue;
        short st = -1;
        if (!un) {
            st = (short)best;
            const float4 a = cd[2 * c];
            const V3 x = v3(a.x, a.y, a.z);
            const int id = cidx(cd, c);
            const V3 pa = pvec(S.pa, NP, best), t1 = pvec(S.pt1, NP, best);
            const V3 t2 = patch_t2(v3(S.pn4[best].x, S.pn4[best].y, S.pn4[best].z), t1);
            for (int s = 0; s < kSlots; ++s)
                atomicMax(&S.keys[s * NP + best], slot_key(slot_score(s, x, a.w, pa, t1, t2), id));
        } else {
            const int i = i0 + __popc(um & ((1u << lane) - 1u));
            S.kord[i] = ord_f32(cphi(cd, c));
            S.cl[i] = (short)c;
        }
        S.cst[c] = st;
    }
    bsync<kW>();
    // slot winners of this batch publish their data; the unassigned find their depth rank
    for (int c = tid; c < nc; c += NT) {
        const int j = S.cst[c];
        if (j < 0) continue;
        const int id = cidx(cd, c);
        bool won = false;
        for (int s = 0; s < kSlots; ++s) won |= (key_sample(S.keys[s * NP + j]) == id);
        if (won) scratch_put(scr, id, cpos(cd, c), cphi(cd, c), cnrm(cd, c));
    }
    const int m = *S.nun;
    int *order = reinterpret_cast<int *>(S.kord);   // the depth order replaces the keys
    if (m > kRankSort) {   // many: sort (O(m log^2 m) work against the count's O(m^2))
        depth_sort<kW>(S.kord, S.cl, m);
        int oc[kPer];
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const int i = tid + u * NT;
            oc[u] = i < m ? S.cl[i] : 0;
        }
#pragma unroll
        for (int u = 0; u < kPer; ++u) {   // writes kord, which no thread reads any more
            const int i = tid + u * NT;
            if (i < m) order[i] = oc[u];
        }
    } else {
        int rk[kPer], rc[kPer];
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const int i = tid + u * NT;
            rk[u] = i < m ? depth_rank(S.kord, S.cl, m, i) : -1;
            rc[u] = i < m ? S.cl[i] : 0;
        }
        bsync<kW>();
#pragma unroll
        for (int u = 0; u < kPer; ++u)
            if (rk[u] >= 0) order[rk[u]] = rc[u];
    }
    bsync<kW>();
    // ---- rounds of FindDeepest, BinReduce, AddPatch
    int pos = 0, ns_prev = 0;
    for (;;) {
        if (tid < 32) {
            add_patches(S, NP, T0, ns_prev, max_patches, scr);
            pos = next_seeds(S, NP, T0, cd, order, m, pos, cos_patch);
        }
        bsync<kW>();
        const int ns = *S.nseed;
        if (ns == 0) break;
        // BinReduce: every unassigned candidate joins the first seed (in depth order) whose
        // normal is similar enough; slot keys go straight into that patch's keys
        for (int c = tid; c < nc; c += NT) {
            if (S.cst[c] != -1) continue;
            const V3 n = cnrm(cd, c);
            unsigned hit = 0u;   // seeds whose patch c may join
#pragma unroll 4
            for (int u = 0; u < ns; ++u)
                hit |= (unsigned)(c == S.win[u] || ndot(n, S.pn4[T0 + u]) >= cos_patch) << u;
            if (hit == 0u) continue;
            const int t = __ffs(hit) - 1;
            S.cst[c] = (short)(-4 - t);
            const int T = T0 + t;
            const float4 a = cd[2 * c];
            const int id = cidx(cd, c);
            const V3 pa = pvec(S.pa, NP, T), t1 = pvec(S.pt1, NP, T);
            const V3 t2 = patch_t2(v3(S.pn4[T].x, S.pn4[T].y, S.pn4[T].z), t1);
            for (int s = 0; s < kSlots; ++s)
                atomicMax(&S.keys[s * NP + T], slot_key(slot_score(s, v3(a.x, a.y, a.z), a.w, pa, t1, t2), id));
        }
        bsync<kW>();
        // the thread holding a winner publishes its data
        for (int c = tid; c < nc; c += NT) {
            const int st = S.cst[c];
            if (st > -4) continue;
            const int T = T0 + (-4 - st);
            const int id = cidx(cd, c);
            bool won = false;
            for (int s = 0; s < kSlots; ++s) won |= (key_sample(S.keys[s * NP + T]) == id);
            if (won) scratch_put(scr, id, cpos(cd, c), cphi(cd, c), cnrm(cd, c));
            S.cst[c] = -3;   // consumed
        }
        bsync<kW>();
        ns_prev = ns;
    }
    if (tid == 0) *S.nun = 0;
    bsync<kW>();
}

// Writes the reduced contacts of the pair: patches in order, distinct slot members in
// slot order.  Executed by all 32 * kW threads, one patch per thread: each finds its
// patch's distinct members, a block-wide prefix sum over the patches places them.
template <int kW>
__device__ void emit_contacts(const PatchSm &S, int NP, const float4 *scr, DContact *out, int cap, int *count,
                              unsigned *status) {
    constexpr int NT = 32 * kW;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int npat = *S.npat;
    int base = 0;   // contacts of the patches before this chunk
    for (int j0 = 0; j0 < npat; j0 += NT) {
        const int j = j0 + tid;
        int ids[kSlots];
        unsigned dm = 0u;   // slots holding a member not held by an earlier slot
        if (j < npat) {
#pragma unroll
            for (int q = 0; q < kSlots; ++q) {
                ids[q] = key_sample(S.keys[q * NP + j]);
                bool dup = false;
#pragma unroll
                for (int t = 0; t < q; ++t) dup |= (ids[t] == ids[q]);
                if (!dup) dm |= 1u << q;
            }
        }
        const int d = __popc(dm);
        int incl = d;   // inclusive prefix sum over the block's patches
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        int before = 0, total = 0;
        if (kW > 1) {
            if (lane == 31) S.win[warp] = incl;
            bsync<kW>();
            for (int w = 0; w < kW; ++w) {
                const int v = S.win[w];
                before += (w < warp) ? v : 0;
                total += v;
            }
            bsync<kW>();
        } else {
            total = __shfl_sync(0xffffffffu, incl, 31);
        }
        int k = base + before + incl - d;
#pragma unroll
        for (int q = 0; q < kSlots; ++q) {
            if (!((dm >> q) & 1u)) continue;
            if (k < cap) {
                const int id = ids[q];
                const float4 a = scr[2 * id], b = scr[2 * id + 1];
                DContact c;
                c.xa[0] = a.x; c.xa[1] = a.y; c.xa[2] = a.z; c.phi = a.w;
                c.n[0] = b.x; c.n[1] = b.y; c.n[2] = b.z;
                c.sample_patch = id | (j << 24);
                out[k] = c;
            }
            ++k;
        }
        base += total;
    }
    if (tid == 0) {
        if (base > cap) atomicOr(status, kStatusOverflow);
        *count = base < cap ? base : cap;
    }
}

// Stages candidates [start, end) of a caller's list (fw_candidate layout: sample, phi,
// x[3], n[3]) in the batch layout.
template <int kW>
__device__ __forceinline__ void load_list(float4 *stage, const float *cands, int start, int end) {
    const int *ci = reinterpret_cast<const int *>(cands);
    for (int c = start + (int)threadIdx.x; c < end; c += 32 * kW) {
        const float *r = cands + 8 * c;
        stage[2 * (c - start)] = make_float4(r[2], r[3], r[4], r[1]);
        stage[2 * (c - start) + 1] = make_float4(r[5], r[6], r[7], __int_as_float(ci[8 * c]));
    }
    bsync<kW>();
}

// ---------------------------------------------------------------------------------------
// kThr threads per CTA (per-sample generation: 128, 256 or 512, chosen by the detection
// autotuner; each thread queries kBatch / kThr samples; per-triangle generation: 256).
// Resident blocks per SM the query kernel is compiled for.  Per-sample lookups wait on the
// cell loads (L2 hits): five 256-thread blocks (48 registers a thread, a 20-byte spill) ran
// 6.6% faster than four (64 registers) at 1000 nut-bolt envs, six (40 registers, more
// spills) 2%.  Per-triangle generation keeps four (its 32 KB of face results per block).
constexpr int query_min_blocks(bool tri, int thr) { return tri ? 1024 / thr : (thr <= 256 ? 5 : 1024 / thr); }

template <bool kTri, int kStore, int kThr, bool kCull = false>
__global__ void __launch_bounds__(kThr, query_min_blocks(kTri, kThr)) query_kernel(SimParams p) {
    static_assert(!kTri || kThr == kQueryThreads, "per-triangle generation runs 256 threads");
    static_assert(!kCull || (!kTri && kStore == kStoreDense), "the cull is of dense per-sample queries");
    constexpr int NPER = kBatch / kThr, NW = kThr / 32;
    const int item = blockIdx.x;
    // pile launches cover every pile's item region; items past a pile's count do nothing
    if (p.pile_counts && item % p.pile_icap >= p.pile_counts[item / p.pile_icap].y) return;
    const int2 it = p.items[item];
    const int pi = it.x, base = it.y * kBatch;
    const PairDev P = p.pairs[pi];
    const AssetDev ga = p.assets[P.asset_a];
    const AssetDev gb = p.assets[P.asset_b];
    // Broad phase: when the bodies' bounding spheres (about their origins, over every vertex
    // and sample) are farther apart than the contact offset plus two voxels of the SDF, no
    // point of A can come closer than that to B's surface, and the interpolated SDF is
    // within sqrt(3) voxels of the distance: the item has no candidate.
    if (p.broad_phase) {   // worlds whose envs hold several pairs
        const V3 dp = ld3(p.pos + 3 * P.a) - ld3(p.pos + 3 * P.b);
        const float lim = ga.radius + gb.radius + p.contact_offset + 2.0f * gb.h;
        if (dot(dp, dp) > lim * lim) {   // the same for every thread of the block
            if (threadIdx.x == 0) p.cand_count[item] = 0;
            return;
        }
    }
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const float cutoff = p.contact_offset;
    V3 xw[NPER], nw[NPER];
    float ph[NPER];
    bool ok[NPER];
    if (kTri) {   // one candidate per triangle of the mesh, the pose shared in shared memory
        __shared__ PairXf Xs;
        __shared__ float4 tres[2 * kBatch];
        if (tid == 0) {
            load_pose(p, P.a, Xs.RA, Xs.pA);
            load_pose(p, P.b, Xs.RB, Xs.pB);
        }
        __syncthreads();
        const unsigned okb = tri_batch<kStore>(Xs, ga, gb, base, tid, p.tri_iters, cutoff, tres);
#pragma unroll
        for (int u = 0; u < NPER; ++u) {   // the thread's own results
            ok[u] = (okb >> u) & 1u;
            const float4 r0 = tres[2 * (u * kThr + tid)], r1 = tres[2 * (u * kThr + tid) + 1];
            xw[u] = v3(r0.x, r0.y, r0.z);
            ph[u] = r0.w;
            nw[u] = v3(r1.x, r1.y, r1.z);
        }
    } else {      // one per surface sample, through the pair's map (map_kernel)
        const PairMap M = p.maps[pi];
        PairXf X;
        load_pose(p, P.a, X.RA, X.pA);
        load_pose(p, P.b, X.RB, X.pB);
        // the cull (fw_set_query_cull): the warp's kCullGroup consecutive samples of a round
        // are skipped when map_cull_kernel set their bit in the item's mask (a separate
        // instantiation: the skip's branches cost the loop time where nothing is culled)
        static_assert(kCullGroup == 32 && kThr % 32 == 0, "a cull group is one warp's round");
        const unsigned cmask = kCull ? __ldg(&p.cull_mask[item]) : 0u;
#pragma unroll
        for (int u = 0; u < NPER; ++u) {
            const int i = base + u * kThr + tid;
            if (kCull && ((cmask >> ((u * kThr) / kCullGroup + warp)) & 1u)) {   // the same on every lane
                ok[u] = false;
                continue;
            }
            const float4 s = __ldg(&ga.samples[i < ga.ns ? i : ga.ns - 1]);
            ok[u] = query_sample<kStore>(M, X, gb, s, cutoff, xw[u], nw[u], ph[u]) && (i < ga.ns);
        }
    }
    // compaction in sample order: local sample u * kThr + warp * 32 + lane
    __shared__ int cnt[NPER * NW];
    unsigned m[NPER];
#pragma unroll
    for (int u = 0; u < NPER; ++u) {
        m[u] = __ballot_sync(0xffffffffu, ok[u]);
        if (lane == 0) cnt[u * NW + warp] = __popc(m[u]);
    }
    __syncthreads();
    // offsets: an exclusive scan of the NPER * NW = 32 counts in (round, warp) order, by
    // every warp for itself (lane l holds count l; shuffles, no further barrier)
    static_assert(NPER * NW == 32, "one count per lane");
    const int cl = cnt[lane];
    int incl = cl;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const int excl = incl - cl;
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    int off[NPER];
#pragma unroll
    for (int u = 0; u < NPER; ++u) off[u] = __shfl_sync(0xffffffffu, excl, u * NW + warp);
    float4 *out = p.cand + (size_t)item * 2 * kBatch;
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int u = 0; u < NPER; ++u) {
        if (ok[u]) {
            const int k = off[u] + __popc(m[u] & lt);
            out[2 * k] = make_float4(xw[u].x, xw[u].y, xw[u].z, ph[u]);
            out[2 * k + 1] = make_float4(nw[u].x, nw[u].y, nw[u].z, __int_as_float(base + u * kThr + tid));
        }
    }
    if (tid == 0) p.cand_count[item] = total;
}

template <int kW>
__global__ void __launch_bounds__(32 * kW, kW >= 8 ? 4 : 8) reduce_kernel(SimParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int pi = blockIdx.x;
    if (p.pile_counts && pi % p.pile_pcap >= p.pile_counts[pi / p.pile_pcap].x) return;
    const int NP = p.max_patches + kWin;
    const PatchSm S = carve_patch(smem_raw, NP);
    float4 *stage = reinterpret_cast<float4 *>(smem_raw + patch_smem_bytes(NP));
    init_patches<kW>(S, NP);
    float4 *scr = p.scratch + p.pairs[pi].scratch_off;
    const int i0 = p.item_range ? p.item_range[pi].x : p.pair_item0[pi];
    const int i1 = p.item_range ? p.item_range[pi].y : p.pair_item0[pi + 1];
    for (int it = i0; it < i1; ++it) {
        const int nc = p.cand_count[it];
        if (nc == 0) continue;
        const float4 *cd = p.cand + (size_t)it * 2 * kBatch;
        if (nc <= kStage) {
            for (int k = threadIdx.x; k < 2 * nc; k += 32 * kW) stage[k] = cd[k];
            bsync<kW>();
            cd = stage;
        }
        reduce_batch<kW>(S, NP, cd, nc, p.max_patches, p.cos_patch, scr);
    }
    emit_contacts<kW>(S, NP, scr, p.contacts + (long long)pi * p.cap_pair, p.cap_pair, p.counts + pi, p.status);
}

// Algorithm 1 on a candidate list in global memory (fw_candidate layout, sorted by
// sample) -- the same reduction code as reduce_kernel, for parity tests.
template <int kW>
__global__ void __launch_bounds__(32 * kW) reduce_list_kernel(SimParams p, const float *cands, int n, float4 *scr,
                                                              DContact *out, int cap, int *count, int *npatch) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int NP = p.max_patches + kWin;
    const PatchSm S = carve_patch(smem_raw, NP);
    float4 *stage = reinterpret_cast<float4 *>(smem_raw + patch_smem_bytes(NP));
    init_patches<kW>(S, NP);
    const int *ci = reinterpret_cast<const int *>(cands);
    int start = 0;
    while (start < n) {
        const int bidx = ci[8 * start] / kBatch;
        int end = start;
        while (end < n && ci[8 * end] / kBatch == bidx) ++end;
        load_list<kW>(stage, cands, start, end);
        reduce_batch<kW>(S, NP, stage, end - start, p.max_patches, p.cos_patch, scr);
        start = end;
    }
    emit_contacts<kW>(S, NP, scr, out, cap, count, p.status);
    if (threadIdx.x == 0) *npatch = *S.npat;
}

__global__ void query_sdf_kernel(AssetDev g, const float *pts, int n, float *phi, float *grad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const V3 x = v3(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
    float f;
    V3 gr;
    if (sdf_lookup_any(g, x, f, gr)) {
        phi[i] = f;
        grad[3 * i] = gr.x; grad[3 * i + 1] = gr.y; grad[3 * i + 2] = gr.z;
    } else {
        phi[i] = __int_as_float(0x7f800000);
        grad[3 * i] = 0.f; grad[3 * i + 1] = 0.f; grad[3 * i + 2] = 0.f;
    }
}

__global__ void tri_pair_kernel(SimParams p, int pi, float *x, float *phi, float *nrm) {
    const PairDev P = p.pairs[pi];
    const AssetDev ga = p.assets[P.asset_a];
    const AssetDev gb = p.assets[P.asset_b];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ga.nt) return;
    PairXf X;
    load_pose(p, P.a, X.RA, X.pA);
    load_pose(p, P.b, X.RB, X.pB);
    V3 xw, nw;
    float f;
    const bool ok = tri_sample(X, ga, gb, t, p.tri_iters, xw, nw, f);
    x[3 * t] = xw.x; x[3 * t + 1] = xw.y; x[3 * t + 2] = xw.z;
    phi[t] = ok ? f : __int_as_float(0x7f800000);
    nrm[3 * t] = ok ? nw.x : 0.f; nrm[3 * t + 1] = ok ? nw.y : 0.f; nrm[3 * t + 2] = ok ? nw.z : 0.f;
}

__global__ void query_pair_kernel(SimParams p, int pi, float *phi, float *nrm) {
    const PairDev P = p.pairs[pi];
    const AssetDev ga = p.assets[P.asset_a];
    const AssetDev gb = p.assets[P.asset_b];
    __shared__ PairMap Ms;
    if (threadIdx.x == 0) pair_map(p, P, gb, Ms);
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ga.ns) return;
    PairXf X;
    load_pose(p, P.a, X.RA, X.pA);
    load_pose(p, P.b, X.RB, X.pB);
    V3 xw, nw;
    float f;
    if (query_sample(Ms, X, gb, ga.samples[i], __int_as_float(0x7f800000), xw, nw, f)) {   // every valid sample
        phi[i] = f;
        nrm[3 * i] = nw.x; nrm[3 * i + 1] = nw.y; nrm[3 * i + 2] = nw.z;
    } else {
        phi[i] = __int_as_float(0x7f800000);
        nrm[3 * i] = 0.f; nrm[3 * i + 1] = 0.f; nrm[3 * i + 2] = 0.f;
    }
}

// ---------------------------------------------------------------------------------------
// Piles (pile envs): the pairs of every pile are found again before each detection.
// Exclusive prefix sum over a block of up to 1024 threads (blockDim a multiple of 32);
// returns the thread's offset, *total the block's sum.
__device__ int block_scan(int v, int *warp_sums, int &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int x = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += u;
        }
        if (lane < nw) warp_sums[lane] = x;   // inclusive over warps
    }
    __syncthreads();
    const int before = warp > 0 ? warp_sums[warp - 1] : 0;
    total = warp_sums[nw - 1];
    __syncthreads();   // warp_sums may be reused by the caller's next scan
    return before + incl - v;
}

// Per-body facts the pair rule of a pile reads, staged in shared memory: position and
// bounding radius, the SDF's voxel size, and flags (movable, has samples, has an SDF).
constexpr unsigned kPileMovable = 1u, kPileSamples = 2u, kPileGrid = 4u;
struct PileStage {
    float4 sph[kMaxPileBodies];
    float h[kMaxPileBodies];
    unsigned char fl[kMaxPileBodies];
};

// Pair rule of a pile for local bodies i < j: i's samples against j's SDF when i has samples
// and j an SDF, else j's samples against i's SDF when j has samples and i an SDF; at least
// one of the two movable; bounding spheres within the contact offset plus two voxels of the
// SDF body (no candidate is possible farther apart).  Returns false for no pair.
__device__ __forceinline__ bool pile_pair_rule(const PileStage &S, float offset, int i, int j, int &a, int &b) {
    const unsigned fi = S.fl[i], fj = S.fl[j];
    if (!((fi | fj) & kPileMovable)) return false;
    if ((fi & kPileSamples) && (fj & kPileGrid)) { a = i; b = j; }
    else if ((fj & kPileSamples) && (fi & kPileGrid)) { a = j; b = i; }
    else return false;
    const float4 A = S.sph[a], Bs = S.sph[b];
    const V3 d = v3(A.x, A.y, A.z) - v3(Bs.x, Bs.y, Bs.z);
    const float lim = A.w + Bs.w + offset + 2.0f * S.h[b];
    return dot(d, d) <= lim * lim;
}

// One block per pile: the pile's pairs in (i, j) order into pairs[pair0 ..], their Generate
// batches into items[item0 ..] and item_range, and counts[pile] = (pairs, items).  More
// pairs or items than the pile's regions hold are dropped and flagged (overflow status).
__global__ void __launch_bounds__(1024) pile_pairs_kernel(SimParams p, const PileDev *piles, PairDev *pairs,
                                                          int2 *items, int2 *item_range, int2 *counts) {
    __shared__ int warp_sums[32];
    __shared__ PileStage S;
    const PileDev P = piles[blockIdx.x];
    const int t = threadIdx.x, n = P.n_bodies, b0 = P.first_body;
    for (int i = t; i < n; i += blockDim.x) {
        const BodyProps &Pi = p.props[b0 + i];
        const AssetDev &Ai = p.assets[Pi.asset];
        const V3 x = ld3(p.pos + 3 * (b0 + i));
        S.sph[i] = make_float4(x.x, x.y, x.z, Ai.radius);
        S.h[i] = Ai.h;
        S.fl[i] = (unsigned char)(((Pi.type == FW_BODY_DYNAMIC || Pi.type == FW_BODY_FIXED_AXIS) ? kPileMovable : 0u) |
                                  (Ai.ns > 0 ? kPileSamples : 0u) | ((Ai.cell32 || Ai.cell16) ? kPileGrid : 0u));
    }
    __syncthreads();
    const float off = p.contact_offset;
    int c = 0;
    if (t < n)
        for (int j = t + 1; j < n; ++j) {
            int a, b;
            c += pile_pair_rule(S, off, t, j, a, b) ? 1 : 0;
        }
    int total;
    int k = block_scan(c, warp_sums, total);
    if (t < n)
        for (int j = t + 1; j < n; ++j) {
            int a, b;
            if (!pile_pair_rule(S, off, t, j, a, b)) continue;
            if (k < P.pcap) {
                PairDev D;
                const BodyProps &Pa = p.props[b0 + a], &Pb = p.props[b0 + b];
                D.a = b0 + a; D.b = b0 + b;
                D.asset_a = Pa.asset; D.asset_b = Pb.asset;
                D.env = P.env;
                D.scratch_off = (P.pair0 + k) * P.stride;
                D.mu = (float)sqrt((double)Pa.mu * (double)Pb.mu);
                D.local_a = a; D.local_b = b;
                D.pad_[0] = D.pad_[1] = D.pad_[2] = 0;
                pairs[P.pair0 + k] = D;
            }
            ++k;
        }
    const int np = total < P.pcap ? total : P.pcap;
    if (t == 0 && total > P.pcap) atomicOr(p.status, kStatusOverflow);
    __syncthreads();   // the pairs are written
    int base = 0;
    for (int c0 = 0; c0 < np; c0 += blockDim.x) {
        const int q = c0 + t;
        int nb = 0;
        if (q < np) {
            const AssetDev &A = p.assets[pairs[P.pair0 + q].asset_a];
            nb = (A.ns + kBatch - 1) / kBatch;
        }
        int chunk;
        const int o = base + block_scan(nb, warp_sums, chunk);
        if (q < np) {
            const int lo = o < P.icap ? o : P.icap, hi = o + nb < P.icap ? o + nb : P.icap;
            item_range[P.pair0 + q] = make_int2(P.item0 + lo, P.item0 + hi);
            for (int u = lo; u < hi; ++u) items[P.item0 + u] = make_int2(P.pair0 + q, u - o);
        }
        base += chunk;
    }
    if (t == 0) {
        if (base > P.icap) atomicOr(p.status, kStatusOverflow);
        counts[blockIdx.x] = make_int2(np, base < P.icap ? base : P.icap);
    }
}

// ---------------------------------------------------------------------------------------
// Allocation-free reduction (fw_reduce_noalloc).  Its scratch lives in g_noalloc below:
// [0, 2*kNoAllocMaxSamples) the per-sample winner lines, then the staged contacts of one
// call, then one float4 of counters.  The kernel first checks the caller's candidates
// (strictly increasing samples below kNoAllocMaxSamples); on failure it only writes
// counts = (-1, 0).
constexpr int kStageF4 = 2 * kMaxPatchesCap * kSlots;   // DContact = 2 float4
constexpr int kNoAllocF4 = 2 * kNoAllocMaxSamples + kStageF4 + 1;

__global__ void __launch_bounds__(32) reduce_noalloc_kernel(SimParams p, const float *cands, int n, float4 *scr,
                                                            fw_contact *out, int cap, int *counts) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int *ci = reinterpret_cast<const int *>(cands);
    bool bad = false;
    for (int i = lane; i < n; i += 32) {
        const int sm = ci[8 * i];
        bad |= sm < 0 || sm >= kNoAllocMaxSamples || (i > 0 && ci[8 * (i - 1)] >= sm);
    }
    if (__any_sync(0xffffffffu, bad)) {
        if (lane == 0) { counts[0] = -1; counts[1] = 0; }
        return;
    }
    const int NP = p.max_patches + kWin;
    const PatchSm S = carve_patch(smem_raw, NP);
    float4 *batch = reinterpret_cast<float4 *>(smem_raw + patch_smem_bytes(NP));
    init_patches<1>(S, NP);
    DContact *stage = reinterpret_cast<DContact *>(scr + 2 * kNoAllocMaxSamples);
    int *stage_count = reinterpret_cast<int *>(scr + 2 * kNoAllocMaxSamples + kStageF4);
    int start = 0;
    while (start < n) {
        const int bidx = ci[8 * start] / kBatch;
        int end = start;
        while (end < n && ci[8 * end] / kBatch == bidx) ++end;
        load_list<1>(batch, cands, start, end);
        reduce_batch<1>(S, NP, batch, end - start, p.max_patches, p.cos_patch, scr);
        start = end;
    }
    emit_contacts<1>(S, NP, scr, stage, p.max_patches * kSlots, stage_count, p.status);
    __syncwarp();
    const int k = *stage_count;
    for (int i = lane; i < k && i < cap; i += 32) {
        const DContact c = stage[i];
        fw_contact o;
        o.sample = c.sample_patch & 0xFFFFFF;
        o.patch = (int)((unsigned)c.sample_patch >> 24);
        o.pair = 0;
        o.phi = c.phi;
        for (int a = 0; a < 3; ++a) {
            o.xa[a] = c.xa[a];
            o.n[a] = c.n[a];
            o.xb[a] = __fsub_rn(c.xa[a], __fmul_rn(c.phi, c.n[a]));   // rounded as fw_reduce's host code
        }
        out[i] = o;
    }
    if (lane == 0) { counts[0] = k; counts[1] = *S.npat; }
}

// shared memory of a reduction block that stages up to `stage` candidates
size_t reduce_smem_bytes(int max_patches, int stage) {
    return patch_smem_bytes(max_patches + kWin) + (size_t)stage * 2 * sizeof(float4);
}

}  // namespace

// The scratch of fw_reduce_noalloc: a fixed 2.2 MB block in every device that loads the
// library, shared by all calls.
static __device__ __align__(256) float4 g_noalloc[kNoAllocF4];

namespace {
float4 *g_noalloc_dev[64];                   // its device address per device ordinal
std::atomic<bool> g_noalloc_ready[64];       // set (release) once g_noalloc_dev[d] is valid
std::mutex g_noalloc_mutex;                  // serialises first calls from several host threads
}  // namespace

// First use on a device (that device current): look up the device address of g_noalloc
// (the host-side name is only a stand-in) and raise the kernel's shared-memory limit.
// Neither step allocates memory.  The address is kept for the process's lifetime (a device
// reset would invalidate it; the header tells callers not to reset).
cudaError_t noalloc_setup(int device) {
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    if (g_noalloc_ready[device].load(std::memory_order_acquire)) return cudaSuccess;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (g_noalloc_ready[device].load(std::memory_order_relaxed)) return cudaSuccess;
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(reduce_noalloc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)reduce_smem_bytes(kMaxPatchesCap, kBatch));
    if (e != cudaSuccess) return e;
    g_noalloc_dev[device] = static_cast<float4 *>(ptr);
    g_noalloc_ready[device].store(true, std::memory_order_release);
    return cudaSuccess;
}

cudaError_t launch_reduce_noalloc(const SimParams &p, int device, const float *d_cands, int n, fw_contact *d_out,
                                  int cap, int *d_counts, cudaStream_t s) {
    cudaError_t e = noalloc_setup(device);
    if (e != cudaSuccess) return e;
    reduce_noalloc_kernel<<<1, 32, reduce_smem_bytes(p.max_patches, kBatch), s>>>(
        p, d_cands, n, g_noalloc_dev[device], d_out, cap, d_counts);
    return cudaGetLastError();
}

template <int kW>
static cudaError_t prepare_reduce(int max_patches) {
    cudaError_t e = cudaFuncSetAttribute(reduce_kernel<kW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)reduce_smem_bytes(max_patches, kStage));
    if (e != cudaSuccess) return e;
    // one reduction block per pair, all resident at once: ask for the largest shared-memory
    // share of the SM's on-chip memory
    return cudaFuncSetAttribute(reduce_kernel<kW>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared);
}

// Raises the kernels' dynamic shared-memory limit (outside any stream capture).
cudaError_t prepare_detect(int max_patches) {
    cudaError_t e = prepare_reduce<2>(max_patches);
    if (e == cudaSuccess) e = prepare_reduce<4>(max_patches);
    if (e == cudaSuccess) e = prepare_reduce<8>(max_patches);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(reduce_list_kernel<kReduceWarps>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)reduce_smem_bytes(max_patches, kBatch));
}

cudaError_t launch_query(const SimParams &p, cudaStream_t s) {
    if (p.n_items == 0) return cudaSuccess;
    // the cull (fw_set_query_cull) over dense storage, per-sample generation
    const bool cull = p.cull && p.cull_mask && !p.sdf_bricks && p.contact_gen == 0;
    if (p.contact_gen == 0) {
        if (cull) map_cull_kernel<<<(p.n_pairs + kCullPairs - 1) / kCullPairs, 32 * kCullPairs, 0, s>>>(p);
        else map_kernel<<<(p.n_pairs + 127) / 128, 128, 0, s>>>(p);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const int qt = p.query_threads > 0 ? p.query_threads : kQueryThreads;
    if (cull) {
        if (qt == 128) query_kernel<false, kStoreDense, 128, true><<<p.n_items, 128, 0, s>>>(p);
        else if (qt == 512) query_kernel<false, kStoreDense, 512, true><<<p.n_items, 512, 0, s>>>(p);
        else query_kernel<false, kStoreDense, 256, true><<<p.n_items, 256, 0, s>>>(p);
        return cudaGetLastError();
    }
    if (p.sdf_bricks) {
        if (p.contact_gen == 1) query_kernel<true, kStoreBricks, kQueryThreads><<<p.n_items, kQueryThreads, 0, s>>>(p);
        else if (qt == 128) query_kernel<false, kStoreBricks, 128><<<p.n_items, 128, 0, s>>>(p);
        else if (qt == 512) query_kernel<false, kStoreBricks, 512><<<p.n_items, 512, 0, s>>>(p);
        else query_kernel<false, kStoreBricks, 256><<<p.n_items, 256, 0, s>>>(p);
    } else {
        if (p.contact_gen == 1) query_kernel<true, kStoreDense, kQueryThreads><<<p.n_items, kQueryThreads, 0, s>>>(p);
        else if (qt == 128) query_kernel<false, kStoreDense, 128><<<p.n_items, 128, 0, s>>>(p);
        else if (qt == 512) query_kernel<false, kStoreDense, 512><<<p.n_items, 512, 0, s>>>(p);
        else query_kernel<false, kStoreDense, 256><<<p.n_items, 256, 0, s>>>(p);
    }
    return cudaGetLastError();
}

cudaError_t launch_tri_pair(const SimParams &p, int pair, float *x, float *phi, float *nrm, cudaStream_t s, int nt) {
    if (nt <= 0) return cudaSuccess;
    tri_pair_kernel<<<(nt + 255) / 256, 256, 0, s>>>(p, pair, x, phi, nrm);
    return cudaGetLastError();
}

cudaError_t launch_pile_pairs(const SimParams &p, const PileDev *piles, int n_piles, PairDev *pairs, int2 *items,
                              int2 *item_range, int2 *counts, cudaStream_t s) {
    if (n_piles <= 0) return cudaSuccess;
    pile_pairs_kernel<<<n_piles, 1024, 0, s>>>(p, piles, pairs, items, item_range, counts);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const SimParams &p, cudaStream_t s) {
    if (p.n_pairs == 0) return cudaSuccess;
    const size_t smem = reduce_smem_bytes(p.max_patches, kStage);
    const int rw = p.reduce_warps > 0 ? p.reduce_warps : kReduceWarps;
    if (rw == 2) reduce_kernel<2><<<p.n_pairs, 64, smem, s>>>(p);
    else if (rw == 8) reduce_kernel<8><<<p.n_pairs, 256, smem, s>>>(p);
    else reduce_kernel<4><<<p.n_pairs, 128, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_detect(const SimParams &p, cudaStream_t s) {
    cudaError_t e = launch_query(p, s);
    if (e != cudaSuccess) return e;
    return launch_reduce(p, s);
}

cudaError_t launch_reduce_list(const SimParams &p, const float *d_cands, int n, DContact *out, int *d_count,
                               int *d_npatch, cudaStream_t s) {
    reduce_list_kernel<kReduceWarps><<<1, 32 * kReduceWarps, reduce_smem_bytes(p.max_patches, kBatch), s>>>(
        p, d_cands, n, p.scratch, out, p.max_patches * kSlots, d_count, d_npatch);
    return cudaGetLastError();
}

cudaError_t launch_query_sdf(const AssetDev &g, const float *pts, int n, float *phi, float *grad,
                             cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    query_sdf_kernel<<<(n + 255) / 256, 256, 0, s>>>(g, pts, n, phi, grad);
    return cudaGetLastError();
}

cudaError_t launch_query_pair(const SimParams &p, int pair, float *phi, float *nrm, cudaStream_t s, int ns) {
    if (ns <= 0) return cudaSuccess;
    query_pair_kernel<<<(ns + 255) / 256, 256, 0, s>>>(p, pair, phi, nrm);
    return cudaGetLastError();
}

}  // namespace fw
