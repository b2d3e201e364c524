// fw_api.cu -- host implementation of the C ABI declared in include/fw.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "fw_internal.h"

using namespace fw;

namespace {

struct AssetHost {
    std::vector<float> V;
    std::vector<int> T;
    std::vector<float> S;   // samples, 3 per point
    double density = 0, mass = 0, com[3] = {0, 0, 0}, I[9] = {0};
    float4 *d_samples = nullptr;
    float4 *d_spheres = nullptr;  // AssetDev::spheres
    float4 *d_tri = nullptr;      // 3 per triangle, asset frame
    bool has_sdf = false;
    float lo[3] = {0, 0, 0}, h = 0;
    int dims[3] = {0, 0, 0};
    float *d_grid = nullptr;
    float4 *d_cell32 = nullptr;   // cell-corner copies (AssetDev), one of them per the world's precision
    uint4 *d_cell16 = nullptr;
    int *d_brick = nullptr;       // narrow-band brick table (AssetDev::brick), null when dense
    int bdims[3] = {0, 0, 0};
    int n_stored = 0;             // bricks kept
    float band = 0;               // metres
    long long cell_bytes = 0;     // bytes of the cell-corner copy
    float radius = 0;             // bounding sphere about the asset origin (vertices and samples)
};

}  // namespace

struct fw_world {
    fw_config cfg;
    cudaStream_t stream = nullptr, cap_stream = nullptr;
    bool own_stream = false;
    std::vector<AssetHost> assets;
    AssetDev *d_assets = nullptr;
    // topology and initial state (host)
    std::vector<BodyProps> props;
    std::vector<PairDev> pairs;
    std::vector<EnvDev> envs;
    std::vector<float> h_pos, h_quat, h_vel, h_ang;
    // device
    BodyProps *d_props = nullptr;
    PairDev *d_pairs = nullptr;
    EnvDev *d_envs = nullptr;
    float *d_pos = nullptr, *d_quat = nullptr, *d_vel = nullptr, *d_ang = nullptr;
    DContact *d_contacts = nullptr;
    int *d_counts = nullptr;
    float4 *d_scratch = nullptr;
    int2 *d_items = nullptr;     // detection work list (pair, batch)
    unsigned *d_cull = nullptr;  // per item: its cull mask (SimParams::cull_mask)
    int *d_pair_item0 = nullptr;
    float4 *d_cand = nullptr;    // candidates of every item
    int *d_cand_count = nullptr;
    PairMap *d_maps = nullptr;   // each pair's composed map into its SDF grid
    int n_items = 0;
    Row *d_rows = nullptr;
    unsigned *d_status = nullptr;
    int dev_bodies = 0;          // bodies whose state is on the device
    bool topo_dirty = true, assets_dirty = true;
    long long scratch_len = 0, rows_len = 0;
    // graph
    cudaGraphExec_t gexec = nullptr;
    int g_sub = -1, g_iters = -1;
    // device limits and the solve's launch shape (0: chosen from the env count)
    int n_sm = 0, max_dyn_smem[4] = {0, 0, 0, 0};
    int solve_groups = 0, solve_warps = 0;
    int lam_rows = 0;   // rows per env whose impulses the solve keeps in shared memory (0: every row)
    int query_threads = 0, reduce_warps = 0;   // detection launch shape (0: the defaults)
    int stall = 0;                             // fw_test_stall
    int no_cull = 0;                           // fw_set_query_cull(0)
    // pile envs (fw_add_pile): one region per pile in each pile buffer, every region of the
    // same size (pile_pcap pairs, pile_icap items, pile_rcap rows)
    std::vector<PileDev> piles;
    int n_regular = 0;           // envs of listed pairs
    int pile_pcap = 0, pile_icap = 0, pile_rcap = 0, pile_stride = 0;
    size_t pile_smem = 0;
    PileDev *d_piles = nullptr;
    PairDev *d_ppairs = nullptr;
    int2 *d_pitems = nullptr, *d_pitem_range = nullptr, *d_pcounts = nullptr;
    unsigned *d_pcull = nullptr;   // per pile item: its cull mask (SimParams::cull_mask)
    DContact *d_pcontacts = nullptr;
    int *d_pccounts = nullptr;   // contacts per pile pair
    float4 *d_pscratch = nullptr, *d_pcand = nullptr;
    int *d_pcand_count = nullptr;
    PairMap *d_pmaps = nullptr;
    float4 *d_prows = nullptr;   // kPileRowF4 float4 per row
    PileSolveMem pmem = {};
    int pile_sweep_blocks = 0;   // blocks of the cooperative pile sweep kernel
    int pile_optin = 0;
    // differentiable rollout (fw_record_rollout .. fw_adjoint_rollout)
    DiffState diff;
    bool diff_valid = false;
    // timing
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<cudaEvent_t> ev_used;   // triples per substep
    std::string err;
};

namespace {

fw_status fail(fw_world *w, fw_status s, const std::string &msg) {
    if (w) w->err = msg;
    return s;
}
fw_status cuda_fail(fw_world *w, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    return fail(w, e == cudaErrorMemoryAllocation ? FW_ERR_OOM : FW_ERR_CUDA, m);
}
#define CK(expr)                                                     \
    do {                                                             \
        cudaError_t e_ = (expr);                                     \
        if (e_ != cudaSuccess) return cuda_fail(w, e_, #expr);       \
    } while (0)

template <class T>
void dfree(T *&p) {
    if (p) cudaFree(p);
    p = nullptr;
}

// ---- mass properties: polyhedral volume integrals of 1, x, y, z, x^2, y^2, z^2, xy, yz,
// zx via the divergence theorem (Eberly, "Polyhedral Mass Properties (Revisited)").
void mass_props(const std::vector<float> &V, const std::vector<int> &T, double density, double &mass,
                double com[3], double I[9]) {
    double in[10] = {0};
    auto sub = [](double w0, double w1, double w2, double &f1, double &f2, double &f3, double &g0, double &g1,
                  double &g2) {
        const double t0 = w0 + w1;
        f1 = t0 + w2;
        const double t1 = w0 * w0;
        const double t2 = t1 + w1 * t0;
        f2 = t2 + w2 * f1;
        f3 = w0 * t1 + w1 * t2 + w2 * f2;
        g0 = f2 + w0 * (f1 + w0);
        g1 = f2 + w1 * (f1 + w1);
        g2 = f2 + w2 * (f1 + w2);
    };
    for (size_t t = 0; t < T.size() / 3; ++t) {
        const float *p0 = &V[3 * T[3 * t]], *p1 = &V[3 * T[3 * t + 1]], *p2 = &V[3 * T[3 * t + 2]];
        const double x0 = p0[0], y0 = p0[1], z0 = p0[2], x1 = p1[0], y1 = p1[1], z1 = p1[2];
        const double x2 = p2[0], y2 = p2[1], z2 = p2[2];
        const double a1 = x1 - x0, b1 = y1 - y0, c1 = z1 - z0, a2 = x2 - x0, b2 = y2 - y0, c2 = z2 - z0;
        const double d0 = b1 * c2 - b2 * c1, d1 = a2 * c1 - a1 * c2, d2 = a1 * b2 - a2 * b1;
        double f1x, f2x, f3x, g0x, g1x, g2x, f1y, f2y, f3y, g0y, g1y, g2y, f1z, f2z, f3z, g0z, g1z, g2z;
        sub(x0, x1, x2, f1x, f2x, f3x, g0x, g1x, g2x);
        sub(y0, y1, y2, f1y, f2y, f3y, g0y, g1y, g2y);
        sub(z0, z1, z2, f1z, f2z, f3z, g0z, g1z, g2z);
        in[0] += d0 * f1x;
        in[1] += d0 * f2x; in[2] += d1 * f2y; in[3] += d2 * f2z;
        in[4] += d0 * f3x; in[5] += d1 * f3y; in[6] += d2 * f3z;
        in[7] += d0 * (y0 * g0x + y1 * g1x + y2 * g2x);
        in[8] += d1 * (z0 * g0y + z1 * g1y + z2 * g2y);
        in[9] += d2 * (x0 * g0z + x1 * g1z + x2 * g2z);
    }
    in[0] /= 6.0;
    for (int k = 1; k <= 3; ++k) in[k] /= 24.0;
    for (int k = 4; k <= 6; ++k) in[k] /= 60.0;
    for (int k = 7; k <= 9; ++k) in[k] /= 120.0;
    const double m = in[0];
    const double cx = in[1] / m, cy = in[2] / m, cz = in[3] / m;
    const double Ixx = in[5] + in[6] - m * (cy * cy + cz * cz);
    const double Iyy = in[4] + in[6] - m * (cz * cz + cx * cx);
    const double Izz = in[4] + in[5] - m * (cx * cx + cy * cy);
    const double Ixy = -(in[7] - m * cx * cy);
    const double Iyz = -(in[8] - m * cy * cz);
    const double Ixz = -(in[9] - m * cz * cx);
    mass = m * density;
    com[0] = cx; com[1] = cy; com[2] = cz;
    const double M[9] = {Ixx, Ixy, Ixz, Ixy, Iyy, Iyz, Ixz, Iyz, Izz};
    for (int k = 0; k < 9; ++k) I[k] = M[k] * density;
}

bool inv3(const double A[9], double B[9]) {
    const double c0 = A[4] * A[8] - A[5] * A[7], c1 = A[5] * A[6] - A[3] * A[8], c2 = A[3] * A[7] - A[4] * A[6];
    const double det = A[0] * c0 + A[1] * c1 + A[2] * c2;
    if (!(std::fabs(det) > 0)) return false;
    const double id = 1.0 / det;
    B[0] = c0 * id; B[3] = c1 * id; B[6] = c2 * id;
    B[1] = (A[2] * A[7] - A[1] * A[8]) * id; B[4] = (A[0] * A[8] - A[2] * A[6]) * id; B[7] = (A[1] * A[6] - A[0] * A[7]) * id;
    B[2] = (A[1] * A[5] - A[2] * A[4]) * id; B[5] = (A[2] * A[3] - A[0] * A[5]) * id; B[8] = (A[0] * A[4] - A[1] * A[3]) * id;
    return true;
}

// ---- grid placement: padded bounding box; h = fl32(L / (res - 1)) with L the longest
// padded extent; lo_a = fl32(centre_a - h (dims_a - 1) / 2)
void grid_placement(const std::vector<float> &V, int res, float pad, int cubic, float lo[3], float &h, int dims[3]) {
    double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
    for (size_t i = 0; i < V.size() / 3; ++i)
        for (int a = 0; a < 3; ++a) {
            mn[a] = std::min(mn[a], (double)V[3 * i + a]);
            mx[a] = std::max(mx[a], (double)V[3 * i + a]);
        }
    double ext[3], L = 0;
    for (int a = 0; a < 3; ++a) {
        ext[a] = (mx[a] - mn[a]) + 2.0 * (double)pad;
        L = std::max(L, ext[a]);
    }
    h = (float)(L / (double)(res - 1));
    for (int a = 0; a < 3; ++a) {
        dims[a] = cubic ? res : (int)std::ceil(ext[a] / (double)h - 1e-9) + 1;
        lo[a] = (float)(0.5 * (mn[a] + mx[a]) - (double)h * (double)(dims[a] - 1) * 0.5);
    }
}

AssetDev asset_view(const AssetHost &A, bool fp16) {
    AssetDev g;
    memset(&g, 0, sizeof g);
    g.samples = A.d_samples;
    g.spheres = A.d_spheres;
    g.ns = (int)(A.S.size() / 3);
    g.tri = A.d_tri;
    g.nt = (int)(A.T.size() / 3);
    g.grid = A.d_grid;
    g.cell32 = fp16 ? nullptr : A.d_cell32;
    g.cell16 = fp16 ? A.d_cell16 : nullptr;
    g.brick = A.d_brick;
    for (int a = 0; a < 3; ++a) g.bdims[a] = A.bdims[a];
    g.band = A.band;
    g.radius = A.radius;
    for (int a = 0; a < 3; ++a) { g.lo[a] = A.lo[a]; g.dims[a] = A.dims[a]; }
    g.h = A.h;
    const double ih = A.h > 0 ? 1.0 / (double)A.h : 0.0;
    g.inv_h = (float)ih;
    g.inv_h_lo = (float)(ih - (double)g.inv_h);
    return g;
}

void drop_graph(fw_world *w) {
    if (w->gexec) cudaGraphExecDestroy(w->gexec);
    w->gexec = nullptr;
}

fw_status upload_assets(fw_world *w) {
    if (!w->assets_dirty) return FW_OK;
    std::vector<AssetDev> v;
    for (auto &A : w->assets) v.push_back(asset_view(A, w->cfg.sdf_fp16 != 0));
    dfree(w->d_assets);
    if (!v.empty()) {
        CK(cudaMalloc(&w->d_assets, sizeof(AssetDev) * v.size()));
        CK(cudaMemcpy(w->d_assets, v.data(), sizeof(AssetDev) * v.size(), cudaMemcpyHostToDevice));
    }
    w->assets_dirty = false;
    drop_graph(w);
    return FW_OK;
}

int cap_pair(const fw_world *w) { return w->cfg.max_patches * kSlots; }

// candidate sources of a pair's point body: its samples, or its triangles
long long pair_sources(const fw_world *w, int asset_a) {
    const AssetHost &A = w->assets[asset_a];
    return (long long)(w->cfg.contact_gen == 1 ? A.T.size() / 3 : A.S.size() / 3);
}

// pairs a pile found in its last detection (synchronises)
fw_status pile_pair_count(fw_world *w, int pile, int *n) {
    int2 c = make_int2(0, 0);
    CK(cudaMemcpyAsync(&c, w->d_pcounts + pile, sizeof c, cudaMemcpyDeviceToHost, w->stream));
    CK(cudaStreamSynchronize(w->stream));
    *n = c.x;
    return FW_OK;
}

void pile_free(fw_world *w) {
    dfree(w->d_piles); dfree(w->d_ppairs); dfree(w->d_pitems); dfree(w->d_pitem_range); dfree(w->d_pcounts);
    dfree(w->d_pcontacts); dfree(w->d_pccounts); dfree(w->d_pscratch); dfree(w->d_pcand); dfree(w->d_pcand_count);
    dfree(w->d_pmaps); dfree(w->d_prows); dfree(w->d_pcull);
    dfree(w->pmem.color); dfree(w->pmem.ab); dfree(w->pmem.rr); dfree(w->pmem.order); dfree(w->pmem.cstart);
    dfree(w->pmem.ncol); dfree(w->pmem.bv); dfree(w->pmem.bw); dfree(w->pmem.bcom); dfree(w->pmem.binv); dfree(w->pmem.bar);
}

// The pile buffers: every pile gets regions of the same size, from the largest pile's
// capacities (pairs, rows) and the largest sample count among the piles' bodies (the
// per-pair winner scratch and the Generate batches per pair).
fw_status pile_alloc(fw_world *w) {
    pile_free(w);
    const int n = (int)w->piles.size();
    if (n == 0) return FW_OK;
    int pcap = 1, rcap = 1, nb_max = 1;
    long long ns_max = 1;
    for (const PileDev &P : w->piles) {
        pcap = std::max(pcap, P.pcap);
        rcap = std::max(rcap, P.rcap);
        nb_max = std::max(nb_max, P.n_bodies);
        for (int i = 0; i < P.n_bodies; ++i)
            ns_max = std::max(ns_max, (long long)w->assets[w->props[P.first_body + i].asset].S.size() / 3);
    }
    const long long icap = (long long)pcap * ((ns_max + kBatch - 1) / kBatch);
    if (icap * n > 0x7FFFFFFFLL || 2 * ns_max * pcap * n > 0x7FFFFFFFLL || (long long)rcap * n > 0x7FFFFFFFLL)
        return fail(w, FW_ERR_ARG, "pile buffers: too many pairs, samples or rows");
    if (pile_smem_bytes(nb_max, pcap) > (size_t)w->pile_optin)
        return fail(w, FW_ERR_ARG, "pile buffers: the piles do not fit the solve's shared memory together");
    w->pile_pcap = pcap;
    w->pile_rcap = rcap;
    w->pile_icap = (int)icap;
    w->pile_stride = (int)(2 * ns_max);
    w->pile_smem = pile_smem_bytes(nb_max, pcap);
    std::vector<PileDev> dev = w->piles;
    for (int k = 0; k < n; ++k) {
        PileDev &P = dev[k];
        P.pair0 = k * pcap; P.pcap = pcap;
        P.item0 = k * w->pile_icap; P.icap = w->pile_icap;
        P.row0 = k * rcap; P.rcap = rcap;
        P.stride = w->pile_stride;
    }
    const size_t np = (size_t)n * pcap, ni = (size_t)n * w->pile_icap;
    CK(cudaMalloc(&w->d_piles, sizeof(PileDev) * n));
    CK(cudaMemcpy(w->d_piles, dev.data(), sizeof(PileDev) * n, cudaMemcpyHostToDevice));
    CK(cudaMalloc(&w->d_ppairs, sizeof(PairDev) * np));
    CK(cudaMalloc(&w->d_pmaps, sizeof(PairMap) * np));
    CK(cudaMalloc(&w->d_pitem_range, sizeof(int2) * np));
    CK(cudaMalloc(&w->d_pccounts, sizeof(int) * np));
    CK(cudaMalloc(&w->d_pcontacts, sizeof(DContact) * np * cap_pair(w)));
    CK(cudaMalloc(&w->d_pscratch, sizeof(float4) * np * w->pile_stride));
    CK(cudaMalloc(&w->d_pitems, sizeof(int2) * ni));
    CK(cudaMalloc(&w->d_pcull, sizeof(unsigned) * ni));
    CK(cudaMalloc(&w->d_pcand, sizeof(float4) * 2 * (size_t)kBatch * ni));
    CK(cudaMalloc(&w->d_pcand_count, sizeof(int) * ni));
    CK(cudaMalloc(&w->d_pcounts, sizeof(int2) * n));
    CK(cudaMalloc(&w->d_prows, sizeof(float4) * kPileRowF4 * (size_t)n * rcap));
    CK(cudaMalloc(&w->pmem.color, np));
    CK(cudaMalloc(&w->pmem.ab, sizeof(unsigned) * np));
    CK(cudaMalloc(&w->pmem.rr, sizeof(unsigned) * np));
    CK(cudaMalloc(&w->pmem.order, sizeof(int) * np));
    CK(cudaMalloc(&w->pmem.cstart, sizeof(int) * n * (kMaxColors + 1)));
    CK(cudaMalloc(&w->pmem.ncol, sizeof(int) * n));
    const size_t nb = std::max<size_t>(w->props.size(), 1);
    CK(cudaMalloc(&w->pmem.bv, sizeof(float4) * nb));
    CK(cudaMalloc(&w->pmem.bw, sizeof(float4) * nb));
    CK(cudaMalloc(&w->pmem.bcom, sizeof(float4) * nb));
    CK(cudaMalloc(&w->pmem.binv, 2 * sizeof(float4) * nb));
    CK(cudaMalloc(&w->pmem.bar, sizeof(unsigned)));
    // no pairs and no contacts until the first detection
    CK(cudaMemsetAsync(w->d_pcounts, 0, sizeof(int2) * n, w->stream));
    CK(cudaMemsetAsync(w->d_pccounts, 0, sizeof(int) * np, w->stream));
    CK(cudaMemsetAsync(w->d_pcand_count, 0, sizeof(int) * ni, w->stream));
    CK(cudaMemsetAsync(w->pmem.color, 0xFF, np, w->stream));
    return FW_OK;
}

// (Re)builds the device copies of the topology, keeping the device state of bodies that
// are already there.
fw_status ensure_device(fw_world *w) {
    fw_status st = upload_assets(w);
    if (st != FW_OK) return st;
    if (!w->topo_dirty) return FW_OK;
    const int nb = (int)w->props.size();
    if (w->dev_bodies > 0) {   // keep the live state of existing bodies
        CK(cudaStreamSynchronize(w->stream));
        CK(cudaMemcpy(w->h_pos.data(), w->d_pos, sizeof(float) * 3 * w->dev_bodies, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(w->h_quat.data(), w->d_quat, sizeof(float) * 4 * w->dev_bodies, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(w->h_vel.data(), w->d_vel, sizeof(float) * 3 * w->dev_bodies, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(w->h_ang.data(), w->d_ang, sizeof(float) * 3 * w->dev_bodies, cudaMemcpyDeviceToHost));
    }
    dfree(w->d_props); dfree(w->d_pairs); dfree(w->d_envs);
    dfree(w->d_pos); dfree(w->d_quat); dfree(w->d_vel); dfree(w->d_ang);
    dfree(w->d_contacts); dfree(w->d_counts); dfree(w->d_scratch); dfree(w->d_rows);
    dfree(w->d_items); dfree(w->d_pair_item0); dfree(w->d_cand); dfree(w->d_cand_count); dfree(w->d_maps);
    dfree(w->d_cull);
    w->n_items = 0;
    const int np = (int)w->pairs.size(), ne = (int)w->envs.size();
    const int cp = cap_pair(w);
    if (nb > 0) {
        CK(cudaMalloc(&w->d_props, sizeof(BodyProps) * nb));
        CK(cudaMemcpy(w->d_props, w->props.data(), sizeof(BodyProps) * nb, cudaMemcpyHostToDevice));
        CK(cudaMalloc(&w->d_pos, sizeof(float) * 3 * nb));
        CK(cudaMalloc(&w->d_quat, sizeof(float) * 4 * nb));
        CK(cudaMalloc(&w->d_vel, sizeof(float) * 3 * nb));
        CK(cudaMalloc(&w->d_ang, sizeof(float) * 3 * nb));
        CK(cudaMemcpy(w->d_pos, w->h_pos.data(), sizeof(float) * 3 * nb, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(w->d_quat, w->h_quat.data(), sizeof(float) * 4 * nb, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(w->d_vel, w->h_vel.data(), sizeof(float) * 3 * nb, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(w->d_ang, w->h_ang.data(), sizeof(float) * 3 * nb, cudaMemcpyHostToDevice));
    }
    if (np > 0) {
        CK(cudaMalloc(&w->d_pairs, sizeof(PairDev) * np));
        CK(cudaMemcpy(w->d_pairs, w->pairs.data(), sizeof(PairDev) * np, cudaMemcpyHostToDevice));
        CK(cudaMalloc(&w->d_contacts, sizeof(DContact) * (size_t)np * cp));
        CK(cudaMalloc(&w->d_counts, sizeof(int) * np));
        CK(cudaMalloc(&w->d_maps, sizeof(PairMap) * np));
        CK(cudaMemsetAsync(w->d_counts, 0, sizeof(int) * np, w->stream));
        long long sl = 0;
        for (auto &P : w->pairs) sl = std::max(sl, (long long)P.scratch_off + 2LL * pair_sources(w, P.asset_a));
        w->scratch_len = std::max(sl, 2LL);
        CK(cudaMalloc(&w->d_scratch, sizeof(float4) * w->scratch_len));
        // work list: one item per (pair, Generate batch)
        std::vector<int2> items;
        std::vector<int> item0(np + 1, 0);
        for (int pi = 0; pi < np; ++pi) {
            item0[pi] = (int)items.size();
            const long long ns = pair_sources(w, w->pairs[pi].asset_a);
            for (long long b = 0; b * kBatch < ns; ++b) items.push_back(make_int2(pi, (int)b));
        }
        item0[np] = (int)items.size();
        w->n_items = (int)items.size();
        CK(cudaMalloc(&w->d_pair_item0, sizeof(int) * (np + 1)));
        CK(cudaMemcpy(w->d_pair_item0, item0.data(), sizeof(int) * (np + 1), cudaMemcpyHostToDevice));
        if (w->n_items > 0) {
            CK(cudaMalloc(&w->d_items, sizeof(int2) * w->n_items));
            CK(cudaMemcpy(w->d_items, items.data(), sizeof(int2) * w->n_items, cudaMemcpyHostToDevice));
            CK(cudaMalloc(&w->d_cand, sizeof(float4) * 2 * (size_t)kBatch * w->n_items));
            CK(cudaMalloc(&w->d_cand_count, sizeof(int) * w->n_items));
            CK(cudaMalloc(&w->d_cull, sizeof(unsigned) * w->n_items));
        }
    }
    if (ne > 0) {
        // the per-env kernels see a pile env as one without bodies (the pile kernels own it)
        std::vector<EnvDev> dev = w->envs;
        for (EnvDev &E : dev)
            if (E.pile >= 0) { E.n_bodies = 0; E.n_pairs = 0; E.row_cap = 0; E.movable = -1; }
        CK(cudaMalloc(&w->d_envs, sizeof(EnvDev) * ne));
        CK(cudaMemcpy(w->d_envs, dev.data(), sizeof(EnvDev) * ne, cudaMemcpyHostToDevice));
        long long rl = 0;
        for (auto &E : w->envs) rl = std::max(rl, (long long)E.row_off + env_row_span(E));
        w->rows_len = std::max(rl, 1LL);
        CK(cudaMalloc(&w->d_rows, sizeof(Row) * w->rows_len));
    }
    st = pile_alloc(w);
    if (st != FW_OK) return st;
    w->dev_bodies = nb;
    w->topo_dirty = false;
    drop_graph(w);
    return FW_OK;
}

SimParams sim_params(const fw_world *w, float hs, int n_iters) {
    SimParams p;
    memset(&p, 0, sizeof p);
    p.assets = w->d_assets;
    p.pairs = w->d_pairs;
    p.envs = w->d_envs;
    p.props = w->d_props;
    p.pos = w->d_pos; p.quat = w->d_quat; p.linvel = w->d_vel; p.angvel = w->d_ang;
    p.contacts = w->d_contacts;
    p.counts = w->d_counts;
    p.scratch = w->d_scratch;
    p.items = w->d_items;
    p.contact_gen = w->cfg.contact_gen;
    p.sdf_bricks = w->cfg.sdf_band > 0.0f;
    p.multi_movable = 0;
    p.broad_phase = 0;
    for (const auto &E : w->envs) {
        p.multi_movable |= (E.movable == -2);
        p.broad_phase |= (E.n_pairs > 1);
    }
    p.tri_iters = w->cfg.tri_iters;
    p.query_threads = w->query_threads;
    p.stall = w->stall;
    p.cull = !w->no_cull;
    p.cull_mask = w->d_cull;
    p.reduce_warps = w->reduce_warps;
    p.pair_item0 = w->d_pair_item0;
    p.n_items = w->n_items;
    p.cand = w->d_cand;
    p.cand_count = w->d_cand_count;
    p.maps = w->d_maps;
    p.rows = w->d_rows;
    p.status = w->d_status;
    p.n_pairs = (int)w->pairs.size();
    p.n_envs = (int)w->envs.size();
    p.cap_pair = cap_pair(w);
    p.max_patches = w->cfg.max_patches;
    p.contact_offset = w->cfg.contact_offset;
    p.cos_patch = w->cfg.cos_patch;
    p.baumgarte = w->cfg.baumgarte;
    p.max_angvel = w->cfg.max_angvel;
    for (int a = 0; a < 3; ++a) p.gravity[a] = w->cfg.gravity[a];
    p.hs = hs;
    p.n_iters = n_iters;
    p.n_vel_iters = w->cfg.n_vel_iters;
    int rc = 0;
    for (const auto &E : w->envs) rc = std::max(rc, E.row_cap);
    if (w->lam_rows > 0 && w->lam_rows < rc) rc = w->lam_rows;   // envs with more rows: global impulses
    p.lam_cap = rc <= kLamCapMax ? rc : 0;   // larger envs take the general sweep
    p.solver = w->cfg.solver;
    if (p.solver == 1) p.lam_cap = 0;         // Jacobi keeps its impulses in the rows
    return p;
}

// The parameters of the pile launches: the pile buffers in place of the listed pairs'.
SimParams pile_params(const fw_world *w, float hs, int n_iters) {
    SimParams p = sim_params(w, hs, n_iters);
    const int n = (int)w->piles.size();
    p.pairs = w->d_ppairs;
    p.maps = w->d_pmaps;
    p.items = w->d_pitems;
    p.pair_item0 = nullptr;
    p.n_items = n * w->pile_icap;
    p.n_pairs = n * w->pile_pcap;
    p.cand = w->d_pcand;
    p.cand_count = w->d_pcand_count;
    p.contacts = w->d_pcontacts;
    p.counts = w->d_pccounts;
    p.scratch = w->d_pscratch;
    p.rows = nullptr;   // the pile kernels take the pile rows (kPileRowF4 float4 each) as an argument
    p.cull = !w->no_cull;
    p.cull_mask = w->d_pcull;
    p.pile_counts = w->d_pcounts;
    p.item_range = w->d_pitem_range;
    p.pile_pcap = w->pile_pcap;
    p.pile_icap = w->pile_icap;
    p.broad_phase = 0;   // the pile's pair list already holds only pairs within reach
    return p;
}

// detection of every pile: pair list, maps, narrow phase, Algorithm 1
fw_status enqueue_pile_detect(fw_world *w, const SimParams &q, cudaStream_t s) {
    const int n = (int)w->piles.size();
    CK(launch_pile_pairs(q, w->d_piles, n, w->d_ppairs, w->d_pitems, w->d_pitem_range, w->d_pcounts, s));
    CK(launch_query(q, s));
    return FW_OK;
}

SolveShape current_solve_shape(const fw_world *w, const SimParams &p) {
    return solve_shape(p.n_envs, p.lam_cap, w->solve_groups, w->solve_warps, w->max_dyn_smem, w->n_sm);
}

fw_status check_status(fw_world *w) {
    unsigned st = 0;
    CK(cudaMemcpy(&st, w->d_status, sizeof st, cudaMemcpyDeviceToHost));
    if (st) {
        CK(cudaMemsetAsync(w->d_status, 0, sizeof st, w->stream));
        // a wait that gave up comes first: the garbage it leaves may also be non-finite
        if (st & kStatusTimeout) return fail(w, FW_ERR_TIMEOUT, "a bounded device wait gave up");
        if (st & kStatusNonFinite) return fail(w, FW_ERR_NONFINITE, "a body state became non-finite");
        if (st & kStatusOverflow) return fail(w, FW_ERR_OVERFLOW, "a pair produced more contacts, or a pile more pairs or contact rows, than fit");
        if (st & kStatusBounds) return fail(w, FW_ERR_DEVICE_BOUNDS, "device index check failed");
    }
    return FW_OK;
}

cudaEvent_t take_event(fw_world *w) {
    cudaEvent_t e;
    if (!w->ev_pool.empty()) {
        e = w->ev_pool.back();
        w->ev_pool.pop_back();
    } else {
        cudaEventCreate(&e);
    }
    w->ev_used.push_back(e);
    return e;
}

fw_status enqueue_substeps(fw_world *w, cudaStream_t s, int n_substeps, float hs, int n_iters, bool detect,
                           bool timed) {
    SimParams p = sim_params(w, hs, n_iters);
    const SolveShape sh = current_solve_shape(w, p);
    const bool regular = w->n_regular > 0, piles = !w->piles.empty();
    const SimParams q = piles ? pile_params(w, hs, n_iters) : p;
    const int np = (int)w->piles.size();
    for (int k = 0; k < n_substeps; ++k) {
        if (timed) CK(cudaEventRecord(take_event(w), s));
        if (detect && regular) CK(launch_query(p, s));
        if (detect && piles) {
            const fw_status st = enqueue_pile_detect(w, q, s);
            if (st != FW_OK) return st;
        }
        if (timed) CK(cudaEventRecord(take_event(w), s));
        if (detect && regular) CK(launch_reduce(p, s));
        if (detect && piles) CK(launch_reduce(q, s));
        if (timed) CK(cudaEventRecord(take_event(w), s));
        if (regular) CK(launch_solve(p, sh, s));
        if (piles)
            CK(launch_pile_solve(q, w->d_piles, np, w->d_pcounts, w->pmem, w->d_prows, w->pile_smem,
                                 w->pile_sweep_blocks, s));
        if (timed) CK(cudaEventRecord(take_event(w), s));
    }
    return FW_OK;
}

bool ready(fw_world *w) { return w && cudaSetDevice(w->cfg.device) == cudaSuccess; }

void diff_free(fw_world *w) {
    DiffState &d = w->diff;
    dfree(d.dyn); dfree(d.tape_c); dfree(d.tape_n); dfree(d.tape_r); dfree(d.tape_b); dfree(d.ck);
    dfree(d.scratch); dfree(d.rows); dfree(d.rbar); dfree(d.upd); dfree(d.lam); dfree(d.xb); dfree(d.mass_b);
    dfree(d.mu_row); dfree(d.mu_b);
    d = DiffState();
    w->diff_valid = false;
}

// Checks that every env is differentiable (at most one dynamic body, the point body a of
// each of its pairs; no fixed-axis bodies) and returns each env's dynamic body.
fw_status diff_envs(fw_world *w, std::vector<int> &dyn) {
    if (!w->piles.empty()) return fail(w, FW_ERR_ARG, "differentiable rollout: pile envs are not supported");
    dyn.assign(w->envs.size(), -1);
    for (size_t e = 0; e < w->envs.size(); ++e) {
        const EnvDev &E = w->envs[e];
        for (int i = 0; i < E.n_bodies; ++i) {
            const int t = w->props[E.first_body + i].type;
            if (t == FW_BODY_FIXED_AXIS)
                return fail(w, FW_ERR_ARG, "differentiable rollout: fixed-axis bodies are not supported");
            if (t == FW_BODY_DYNAMIC) {
                if (dyn[e] >= 0) return fail(w, FW_ERR_ARG, "differentiable rollout: more than one dynamic body in an env");
                dyn[e] = E.first_body + i;
            }
        }
        for (int k = 0; k < E.n_pairs; ++k)
            if (dyn[e] >= 0 && w->pairs[E.first_pair + k].a != dyn[e])
                return fail(w, FW_ERR_ARG, "differentiable rollout: the dynamic body must be the point body of every pair");
    }
    return FW_OK;
}

template <class T>
fw_status dalloc(fw_world *w, T *&ptr, size_t bytes) {
    dfree(ptr);
    CK(cudaMalloc(reinterpret_cast<void **>(&ptr), bytes > 0 ? bytes : 16));
    return FW_OK;
}

fw_status diff_alloc(fw_world *w, int S, int K) {
    diff_free(w);
    DiffState &d = w->diff;
    const size_t E = w->envs.size(), nb = w->props.size(), np = w->pairs.size();
    int rc = 1;
    for (const auto &en : w->envs) rc = std::max(rc, en.row_cap);
    d.S = S; d.K = K; d.row_cap = rc;
    d.hs = w->cfg.dt / (float)S;
    const size_t slots = (size_t)S * E, rows = E * (size_t)rc;
    fw_status st = FW_OK;
#define DA(ptr, bytes) if ((st = dalloc(w, ptr, bytes)) != FW_OK) return st
    DA(d.dyn, sizeof(int) * E);
    DA(d.tape_c, diff_tape_record_bytes() * slots * rc);
    DA(d.tape_n, sizeof(int) * slots);
    DA(d.tape_r, slots * rc * (size_t)std::max(K, 1));
    DA(d.tape_b, slots);
    DA(d.ck, sizeof(float) * 13 * nb * (size_t)S);
    DA(d.scratch, sizeof(float) * 13 * nb);
    DA(d.rows, diff_row_bytes() * rows);
    DA(d.rbar, diff_row_bar_bytes() * rows);
    DA(d.upd, sizeof(float) * 9 * rows * (size_t)std::max(K, 1));
    DA(d.lam, sizeof(float) * 3 * rows);
    DA(d.xb, sizeof(float) * 13 * nb);
    DA(d.mass_b, sizeof(float) * nb);
    DA(d.mu_row, sizeof(float) * rows);
    DA(d.mu_b, sizeof(float) * std::max(np, (size_t)1));
#undef DA
    CK(cudaMemsetAsync(d.tape_n, 0, sizeof(int) * slots, w->stream));
    return FW_OK;
}

// A body's constant properties from its descriptor (mass scaled from the asset's when the
// descriptor gives one); false when its inertia is singular.
bool body_props(const fw_world *w, const fw_body_desc &d, BodyProps &P) {
    const AssetHost &A = w->assets[d.asset];
    memset(&P, 0, sizeof P);
    P.type = d.type;
    P.asset = d.asset;
    double scale = 1.0, mass = A.mass;
    if (d.mass > 0.0f) { scale = (double)d.mass / A.mass; mass = d.mass; }
    double Ib[9], Ii[9];
    for (int k = 0; k < 9; ++k) Ib[k] = A.I[k] * scale;
    if (!inv3(Ib, Ii)) return false;
    P.mass = (float)mass;
    P.invm = d.type == FW_BODY_DYNAMIC ? (float)(1.0 / mass) : 0.0f;
    for (int a = 0; a < 3; ++a) P.com_b[a] = (float)A.com[a];
    const int sym[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
    for (int k = 0; k < 6; ++k) {
        P.Ib[k] = (float)Ib[3 * sym[k][0] + sym[k][1]];
        P.Ib_inv[k] = (float)Ii[3 * sym[k][0] + sym[k][1]];
    }
    const double an = std::sqrt((double)d.axis[0] * d.axis[0] + (double)d.axis[1] * d.axis[1] +
                                (double)d.axis[2] * d.axis[2]);
    for (int a = 0; a < 3; ++a) {
        P.axis[a] = an > 0 ? (float)(d.axis[a] / an) : 0.0f;
        P.force[a] = d.force[a];
        P.torque[a] = d.torque[a];
    }
    P.mu = d.mu;
    return true;
}

// Appends one validated body: its properties and its initial state (unit quaternion; a
// static body at rest; a fixed-axis body without linear velocity, spinning about its axis).
void append_body(fw_world *w, const fw_body_desc &d) {
    BodyProps P;
    body_props(w, d, P);
    w->props.push_back(P);
    const double qn = std::sqrt((double)d.quat[0] * d.quat[0] + (double)d.quat[1] * d.quat[1] +
                                (double)d.quat[2] * d.quat[2] + (double)d.quat[3] * d.quat[3]);
    for (int a = 0; a < 3; ++a) w->h_pos.push_back(d.pos[a]);
    for (int a = 0; a < 4; ++a) w->h_quat.push_back((float)(d.quat[a] / qn));
    float v[3] = {d.linvel[0], d.linvel[1], d.linvel[2]}, om[3] = {d.angvel[0], d.angvel[1], d.angvel[2]};
    if (d.type == FW_BODY_STATIC) { v[0] = v[1] = v[2] = 0; om[0] = om[1] = om[2] = 0; }
    if (d.type == FW_BODY_FIXED_AXIS) {
        const float s = om[0] * P.axis[0] + om[1] * P.axis[1] + om[2] * P.axis[2];
        v[0] = v[1] = v[2] = 0;
        for (int a = 0; a < 3; ++a) om[a] = s * P.axis[a];
    }
    for (int a = 0; a < 3; ++a) { w->h_vel.push_back(v[a]); w->h_ang.push_back(om[a]); }
}

}  // namespace

// ===================================================================================== ABI
extern "C" {

void fw_config_default(fw_config *c) {
    if (!c) return;
    memset(c, 0, sizeof *c);
    c->gravity[2] = -9.81f;
    c->dt = 1.0f / 60.0f;
    c->contact_offset = 1e-4f;
    c->cos_patch = 0.94f;
    c->max_patches = 128;
    c->patch_dirs = kSlots - 1;
    c->batch_size = kBatch;
    c->baumgarte = 0.2f;
    c->n_vel_iters = 0;
    c->max_angvel = 0.0f;
    c->sdf_fp16 = 0;
    c->contact_gen = 0;
    c->tri_iters = 16;
    c->sdf_band = 0.0f;
    c->solver = 0;
    c->device = 0;
    c->cuda_stream = nullptr;
    c->seed = 0;
}

fw_status fw_create(const fw_config *cfg, fw_world **out) {
    if (!cfg || !out) return FW_ERR_ARG;
    *out = nullptr;
    if (cfg->batch_size != kBatch || cfg->patch_dirs != kSlots - 1 || cfg->max_patches < 1 ||
        cfg->max_patches > kMaxPatchesCap || !(cfg->dt > 0) || cfg->contact_gen < 0 || cfg->contact_gen > 1 ||
        cfg->tri_iters < 0 || cfg->tri_iters > 1024 || !(cfg->sdf_band >= 0.0f && cfg->sdf_band <= 1e6f) ||
        cfg->solver < 0 || cfg->solver > 1)
        return FW_ERR_ARG;
    fw_world *w = new fw_world();
    w->cfg = *cfg;
    cudaError_t e = cudaSetDevice(cfg->device);
    if (e == cudaSuccess && cfg->cuda_stream) w->stream = (cudaStream_t)cfg->cuda_stream;
    if (e == cudaSuccess && !cfg->cuda_stream) {
        e = cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking);
        w->own_stream = (e == cudaSuccess);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&w->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&w->d_status, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(w->d_status, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = prepare_detect(kMaxPatchesCap);   // any later world fits
    int optin = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&w->n_sm, cudaDevAttrMultiProcessorCount, cfg->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, cfg->device);
    if (e == cudaSuccess) e = prepare_solve(optin, w->max_dyn_smem);
    if (e == cudaSuccess) e = prepare_pile_solve(optin, cfg->device, &w->pile_optin, &w->pile_sweep_blocks);
    if (e == cudaSuccess && w->max_dyn_smem[0] < (int)solve_smem_bytes(kLamCapMax)) e = cudaErrorInvalidValue;
    if (e != cudaSuccess) {
        cudaGetLastError();
        fw_destroy(w);
        return e == cudaErrorMemoryAllocation ? FW_ERR_OOM : FW_ERR_CUDA;
    }
    *out = w;
    return FW_OK;
}

fw_status fw_destroy(fw_world *w) {
    if (!w) return FW_OK;
    cudaSetDevice(w->cfg.device);
    if (w->stream) cudaStreamSynchronize(w->stream);
    drop_graph(w);
    diff_free(w);
    for (auto &A : w->assets) {
        dfree(A.d_samples); dfree(A.d_spheres); dfree(A.d_tri); dfree(A.d_grid); dfree(A.d_cell32); dfree(A.d_cell16);
        dfree(A.d_brick);
    }
    dfree(w->d_assets);
    dfree(w->d_props); dfree(w->d_pairs); dfree(w->d_envs);
    dfree(w->d_pos); dfree(w->d_quat); dfree(w->d_vel); dfree(w->d_ang);
    dfree(w->d_contacts); dfree(w->d_counts); dfree(w->d_scratch); dfree(w->d_rows); dfree(w->d_status);
    dfree(w->d_items); dfree(w->d_pair_item0); dfree(w->d_cand); dfree(w->d_cand_count); dfree(w->d_maps);
    dfree(w->d_cull);
    pile_free(w);
    for (auto e : w->ev_pool) cudaEventDestroy(e);
    for (auto e : w->ev_used) cudaEventDestroy(e);
    if (w->cap_stream) cudaStreamDestroy(w->cap_stream);
    if (w->own_stream && w->stream) cudaStreamDestroy(w->stream);
    delete w;
    return FW_OK;
}

fw_status fw_add_mesh_asset(fw_world *w, const float *verts, int n_verts, const int *tris, int n_tris,
                            const float *sample_pts, int n_samples, float density, int *asset_id_out) {
    if (!ready(w)) return FW_ERR_ARG;
    if (!verts || !tris || n_verts < 3 || n_tris < 1 || n_tris > (1 << 24) || n_samples < 0 || n_samples > (1 << 24) ||
        (n_samples > 0 && !sample_pts) || !(density > 0))
        return fail(w, FW_ERR_ARG, "fw_add_mesh_asset: bad argument");
    for (int i = 0; i < 3 * n_tris; ++i)
        if (tris[i] < 0 || tris[i] >= n_verts) return fail(w, FW_ERR_ARG, "fw_add_mesh_asset: triangle index out of range");
    AssetHost A;
    A.V.assign(verts, verts + 3 * n_verts);
    A.T.assign(tris, tris + 3 * n_tris);
    if (n_samples > 0) A.S.assign(sample_pts, sample_pts + 3 * n_samples);
    A.density = density;
    {   // bounding radius, rounded up to float
        double r2 = 0.0;
        for (size_t k = 0; k + 2 < A.V.size(); k += 3)
            r2 = std::max(r2, (double)A.V[k] * A.V[k] + (double)A.V[k + 1] * A.V[k + 1] + (double)A.V[k + 2] * A.V[k + 2]);
        for (size_t k = 0; k + 2 < A.S.size(); k += 3)
            r2 = std::max(r2, (double)A.S[k] * A.S[k] + (double)A.S[k + 1] * A.S[k + 1] + (double)A.S[k + 2] * A.S[k + 2]);
        A.radius = std::nextafter((float)std::sqrt(r2), INFINITY);
    }
    mass_props(A.V, A.T, density, A.mass, A.com, A.I);
    if (!(A.mass > 0)) return fail(w, FW_ERR_ARG, "fw_add_mesh_asset: mesh encloses no volume (winding?)");
    if (n_samples > 0) {
        std::vector<float4> s4(n_samples);
        for (int i = 0; i < n_samples; ++i) s4[i] = make_float4(A.S[3 * i], A.S[3 * i + 1], A.S[3 * i + 2], 0.f);
        CK(cudaMalloc(&A.d_samples, sizeof(float4) * n_samples));
        CK(cudaMemcpy(A.d_samples, s4.data(), sizeof(float4) * n_samples, cudaMemcpyHostToDevice));
        // a bounding sphere per group of kCullGroup consecutive samples: the centre of the
        // group's box, the largest distance to it (float64, then rounded up)
        const int ng = (n_samples + kCullGroup - 1) / kCullGroup;
        std::vector<float4> sp(ng);
        for (int g = 0; g < ng; ++g) {
            double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
            const int i1 = std::min(n_samples, (g + 1) * kCullGroup);
            for (int i = g * kCullGroup; i < i1; ++i)
                for (int a = 0; a < 3; ++a) {
                    mn[a] = std::min(mn[a], (double)A.S[3 * i + a]);
                    mx[a] = std::max(mx[a], (double)A.S[3 * i + a]);
                }
            const float c[3] = {(float)(0.5 * (mn[0] + mx[0])), (float)(0.5 * (mn[1] + mx[1])), (float)(0.5 * (mn[2] + mx[2]))};
            double r2 = 0.0;
            for (int i = g * kCullGroup; i < i1; ++i) {
                double d2 = 0.0;
                for (int a = 0; a < 3; ++a) d2 += ((double)A.S[3 * i + a] - c[a]) * ((double)A.S[3 * i + a] - c[a]);
                r2 = std::max(r2, d2);
            }
            sp[g] = make_float4(c[0], c[1], c[2], std::nextafter((float)std::sqrt(r2), INFINITY));
        }
        CK(cudaMalloc(&A.d_spheres, sizeof(float4) * ng));
        CK(cudaMemcpy(A.d_spheres, sp.data(), sizeof(float4) * ng, cudaMemcpyHostToDevice));
    }
    {   // the faces, for the per-triangle contact generator
        std::vector<float4> t4(3 * (size_t)n_tris);
        for (size_t k = 0; k < t4.size(); ++k)
            t4[k] = make_float4(A.V[3 * A.T[k]], A.V[3 * A.T[k] + 1], A.V[3 * A.T[k] + 2], 0.f);
        CK(cudaMalloc(&A.d_tri, sizeof(float4) * t4.size()));
        CK(cudaMemcpy(A.d_tri, t4.data(), sizeof(float4) * t4.size(), cudaMemcpyHostToDevice));
    }
    w->assets.push_back(std::move(A));
    w->assets_dirty = true;
    if (asset_id_out) *asset_id_out = (int)w->assets.size() - 1;
    return FW_OK;
}

fw_status fw_get_sdf_storage(fw_world *w, int asset_id, long long *cell_bytes, int *bricks_stored, int *bricks_total) {
    if (!w || asset_id < 0 || asset_id >= (int)w->assets.size()) return fail(w, FW_ERR_ARG, "bad asset");
    const AssetHost &A = w->assets[asset_id];
    if (!A.has_sdf) return fail(w, FW_ERR_STATE, "fw_get_sdf_storage: asset has no SDF");
    if (cell_bytes) *cell_bytes = A.cell_bytes;
    if (bricks_stored) *bricks_stored = A.d_brick ? A.n_stored : 0;
    if (bricks_total) *bricks_total = A.d_brick ? A.bdims[0] * A.bdims[1] * A.bdims[2] : 0;
    return FW_OK;
}

fw_status fw_get_mass(fw_world *w, int asset_id, double *mass, double com[3], double inertia[9]) {
    if (!w || asset_id < 0 || asset_id >= (int)w->assets.size()) return fail(w, FW_ERR_ARG, "bad asset");
    const AssetHost &A = w->assets[asset_id];
    if (mass) *mass = A.mass;
    if (com) memcpy(com, A.com, sizeof A.com);
    if (inertia) memcpy(inertia, A.I, sizeof A.I);
    return FW_OK;
}

static fw_status finish_grid(fw_world *w, AssetHost &A) {
    const long long nc = (long long)(A.dims[0] - 1) * (A.dims[1] - 1) * (A.dims[2] - 1);
    const size_t cell = w->cfg.sdf_fp16 ? sizeof(uint4) : 2 * sizeof(float4);
    dfree(A.d_cell32);
    dfree(A.d_cell16);
    dfree(A.d_brick);
    A.n_stored = 0;
    A.band = 0.0f;
    for (int a = 0; a < 3; ++a) A.bdims[a] = 0;
    if (w->cfg.sdf_band > 0.0f) {
        // narrow-band bricks: flag every brick on the device, number the stored ones here,
        // then copy their cells (the dense cell copy is never made)
        A.band = w->cfg.sdf_band * A.h;
        long long nb = 1;
        for (int a = 0; a < 3; ++a) {
            A.bdims[a] = (A.dims[a] - 1 + kBrick - 1) / kBrick;
            nb *= A.bdims[a];
        }
        if (nb > 0x7FFFFFFFLL) return fail(w, FW_ERR_ARG, "narrow-band bricks: grid too large");
        std::vector<int> flag((size_t)nb), of_slot;
        CK(cudaMalloc(&A.d_brick, sizeof(int) * nb));
        CK(launch_brick_flags(A.d_grid, A.dims, A.band, A.bdims, A.d_brick, w->stream));
        CK(cudaMemcpyAsync(flag.data(), A.d_brick, sizeof(int) * nb, cudaMemcpyDeviceToHost, w->stream));
        CK(cudaStreamSynchronize(w->stream));
        for (long long b = 0; b < nb; ++b)
            if (flag[b] == 1) { flag[b] = (int)of_slot.size(); of_slot.push_back((int)b); }
        A.n_stored = (int)of_slot.size();
        CK(cudaMemcpyAsync(A.d_brick, flag.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, w->stream));
        const long long ncs = (long long)(A.n_stored > 0 ? A.n_stored : 1) * kBrickCells;   // >= 1 brick: a valid dummy
        int *d_of_slot = nullptr;
        if (A.n_stored > 0) {
            CK(cudaMalloc(&d_of_slot, sizeof(int) * of_slot.size()));
            CK(cudaMemcpyAsync(d_of_slot, of_slot.data(), sizeof(int) * of_slot.size(), cudaMemcpyHostToDevice,
                               w->stream));
        }
        cudaError_t e;
        if (w->cfg.sdf_fp16) {
            e = cudaMalloc(&A.d_cell16, sizeof(uint4) * ncs);
            if (e == cudaSuccess) e = cudaMemsetAsync(A.d_cell16, 0, sizeof(uint4) * ncs, w->stream);
            if (e == cudaSuccess)
                e = launch_brick_cells(A.d_grid, A.dims, 1.0f / A.h, A.bdims, d_of_slot, A.n_stored, nullptr,
                                       A.d_cell16, w->stream);
        } else {
            e = cudaMalloc(&A.d_cell32, sizeof(float4) * 2 * ncs);
            if (e == cudaSuccess) e = cudaMemsetAsync(A.d_cell32, 0, sizeof(float4) * 2 * ncs, w->stream);
            if (e == cudaSuccess)
                e = launch_brick_cells(A.d_grid, A.dims, 1.0f / A.h, A.bdims, d_of_slot, A.n_stored, A.d_cell32,
                                       nullptr, w->stream);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
        dfree(d_of_slot);
        CK(e);
        A.cell_bytes = (long long)cell * ncs + (long long)sizeof(int) * nb;
    } else if (w->cfg.sdf_fp16) {
        CK(cudaMalloc(&A.d_cell16, sizeof(uint4) * nc));
        CK(launch_cells(A.d_grid, A.dims, 1.0f / A.h, nullptr, A.d_cell16, w->stream));
        A.cell_bytes = (long long)cell * nc;
    } else {
        CK(cudaMalloc(&A.d_cell32, sizeof(float4) * 2 * nc));
        CK(launch_cells(A.d_grid, A.dims, 1.0f / A.h, A.d_cell32, nullptr, w->stream));
        A.cell_bytes = (long long)cell * nc;
    }
    CK(cudaStreamSynchronize(w->stream));
    A.has_sdf = true;
    w->assets_dirty = true;
    return FW_OK;
}

fw_status fw_bake_sdf(fw_world *w, int asset_id, int resolution, float padding_m, int cubic) {
    if (!ready(w)) return FW_ERR_ARG;
    if (asset_id < 0 || asset_id >= (int)w->assets.size() || resolution < 2 || !(padding_m >= 0))
        return fail(w, FW_ERR_ARG, "fw_bake_sdf: bad argument");
    AssetHost &A = w->assets[asset_id];
    grid_placement(A.V, resolution, padding_m, cubic, A.lo, A.h, A.dims);
    const int nt = (int)A.T.size() / 3;
    const int nv = (int)A.V.size() / 3;
    // triangles in Morton order of their centroids, so that shared-memory tiles are compact
    double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
    for (int i = 0; i < nv; ++i)
        for (int a = 0; a < 3; ++a) {
            mn[a] = std::min(mn[a], (double)A.V[3 * i + a]);
            mx[a] = std::max(mx[a], (double)A.V[3 * i + a]);
        }
    auto spread = [](unsigned v) {
        v &= 0x3FF;
        v = (v | (v << 16)) & 0x030000FF;
        v = (v | (v << 8)) & 0x0300F00F;
        v = (v | (v << 4)) & 0x030C30C3;
        v = (v | (v << 2)) & 0x09249249;
        return v;
    };
    std::vector<std::pair<unsigned, int>> order(nt);
    for (int t = 0; t < nt; ++t) {
        unsigned q[3];
        for (int a = 0; a < 3; ++a) {
            const double c = (A.V[3 * A.T[3 * t] + a] + A.V[3 * A.T[3 * t + 1] + a] + A.V[3 * A.T[3 * t + 2] + a]) / 3.0;
            const double u = (c - mn[a]) / std::max(mx[a] - mn[a], 1e-30);
            q[a] = (unsigned)std::min(1023.0, std::max(0.0, std::floor(u * 1023.999)));
        }
        order[t] = {spread(q[0]) | (spread(q[1]) << 1) | (spread(q[2]) << 2), t};
    }
    std::stable_sort(order.begin(), order.end());
    // per triangle: vertices; unit face normal, edge and vertex pseudonormals
    std::vector<double> fn(3 * (size_t)nt);
    std::vector<double> vn(3 * (size_t)nv, 0.0);
    for (int t = 0; t < nt; ++t) {
        const float *p[3] = {&A.V[3 * A.T[3 * t]], &A.V[3 * A.T[3 * t + 1]], &A.V[3 * A.T[3 * t + 2]]};
        double e1[3], e2[3], n[3];
        for (int a = 0; a < 3; ++a) { e1[a] = (double)p[1][a] - p[0][a]; e2[a] = (double)p[2][a] - p[0][a]; }
        n[0] = e1[1] * e2[2] - e1[2] * e2[1]; n[1] = e1[2] * e2[0] - e1[0] * e2[2]; n[2] = e1[0] * e2[1] - e1[1] * e2[0];
        const double l = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        for (int a = 0; a < 3; ++a) fn[3 * t + a] = l > 0 ? n[a] / l : 0.0;
        for (int k = 0; k < 3; ++k) {   // interior angle at corner k
            const float *o = p[k], *u = p[(k + 1) % 3], *v = p[(k + 2) % 3];
            double du[3], dv[3];
            for (int a = 0; a < 3; ++a) { du[a] = (double)u[a] - o[a]; dv[a] = (double)v[a] - o[a]; }
            const double cr[3] = {du[1] * dv[2] - du[2] * dv[1], du[2] * dv[0] - du[0] * dv[2], du[0] * dv[1] - du[1] * dv[0]};
            const double ang = std::atan2(std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]),
                                          du[0] * dv[0] + du[1] * dv[1] + du[2] * dv[2]);
            for (int a = 0; a < 3; ++a) vn[3 * A.T[3 * t + k] + a] += ang * fn[3 * t + a];
        }
    }
    std::map<std::pair<int, int>, int> edge_tri;
    for (int t = 0; t < nt; ++t)
        for (int k = 0; k < 3; ++k) edge_tri[{A.T[3 * t + k], A.T[3 * t + (k + 1) % 3]}] = t;
    std::vector<float> tri(9 * (size_t)nt), pn(21 * (size_t)nt);
    const int ts = bake_tile_size();
    const int ntile = (nt + ts - 1) / ts;
    std::vector<float> box(6 * (size_t)ntile);
    for (int tt = 0; tt < ntile; ++tt)
        for (int a = 0; a < 3; ++a) { box[6 * tt + a] = 3e38f; box[6 * tt + 3 + a] = -3e38f; }
    for (int s = 0; s < nt; ++s) {
        const int t = order[s].second;
        for (int k = 0; k < 3; ++k)
            for (int a = 0; a < 3; ++a) {
                const float c = A.V[3 * A.T[3 * t + k] + a];
                tri[9 * (size_t)s + 3 * k + a] = c;
                float &lo = box[6 * (s / ts) + a], &hi = box[6 * (s / ts) + 3 + a];
                lo = std::min(lo, c);
                hi = std::max(hi, c);
            }
        double nrm[7][3];
        for (int a = 0; a < 3; ++a) nrm[0][a] = fn[3 * t + a];
        for (int k = 0; k < 3; ++k) {   // edges ab, bc, ca: the two adjacent face normals
            const int i0 = A.T[3 * t + k], i1 = A.T[3 * t + (k + 1) % 3];
            auto it = edge_tri.find({i1, i0});
            const int o = (it == edge_tri.end()) ? t : it->second;
            double s3[3], l = 0;
            for (int a = 0; a < 3; ++a) { s3[a] = fn[3 * t + a] + fn[3 * o + a]; l += s3[a] * s3[a]; }
            l = std::sqrt(l);
            for (int a = 0; a < 3; ++a) nrm[1 + k][a] = l > 0 ? s3[a] / l : fn[3 * t + a];
        }
        for (int k = 0; k < 3; ++k) {   // vertices a, b, c: angle-weighted face normals
            const int vi = A.T[3 * t + k];
            const double l = std::sqrt(vn[3 * vi] * vn[3 * vi] + vn[3 * vi + 1] * vn[3 * vi + 1] + vn[3 * vi + 2] * vn[3 * vi + 2]);
            for (int a = 0; a < 3; ++a) nrm[4 + k][a] = l > 0 ? vn[3 * vi + a] / l : fn[3 * t + a];
        }
        for (int q = 0; q < 7; ++q)
            for (int a = 0; a < 3; ++a) pn[21 * (size_t)s + 3 * q + a] = (float)nrm[q][a];
    }
    const long long n_nodes = (long long)A.dims[0] * A.dims[1] * A.dims[2];
    float *d_tri = nullptr, *d_pn = nullptr, *d_box = nullptr;
    int *d_flags = nullptr;
    dfree(A.d_grid);
    dfree(A.d_cell32);
    dfree(A.d_cell16);
    dfree(A.d_brick);
    CK(cudaMalloc(&A.d_grid, sizeof(float) * n_nodes));
    CK(cudaMalloc(&d_tri, sizeof(float) * tri.size()));
    CK(cudaMalloc(&d_pn, sizeof(float) * pn.size()));
    CK(cudaMalloc(&d_box, sizeof(float) * box.size()));
    CK(cudaMalloc(&d_flags, sizeof(int) * (n_nodes + 1)));
    CK(cudaMemcpy(d_tri, tri.data(), sizeof(float) * tri.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_pn, pn.data(), sizeof(float) * pn.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_box, box.data(), sizeof(float) * box.size(), cudaMemcpyHostToDevice));
    CK(cudaMemset(d_flags, 0, sizeof(int)));
    const AssetDev g = asset_view(A, false);
    CK(launch_bake(d_tri, nt, d_pn, d_box, g, A.d_grid, d_flags, w->stream));
    int nflag = 0;
    CK(cudaMemcpyAsync(&nflag, d_flags, sizeof(int), cudaMemcpyDeviceToHost, w->stream));
    CK(cudaStreamSynchronize(w->stream));
    if (nflag > 0) CK(launch_bake_fix_sign(d_tri, nt, g, A.d_grid, d_flags + 1, nflag, w->stream));
    CK(cudaStreamSynchronize(w->stream));
    cudaFree(d_tri); cudaFree(d_pn); cudaFree(d_box); cudaFree(d_flags);
    return finish_grid(w, A);
}

fw_status fw_set_sdf(fw_world *w, int asset_id, const float lo[3], float h, const int dims[3], const float *values) {
    if (!ready(w)) return FW_ERR_ARG;
    if (asset_id < 0 || asset_id >= (int)w->assets.size() || !lo || !dims || !values || !(h > 0) || dims[0] < 2 ||
        dims[1] < 2 || dims[2] < 2)
        return fail(w, FW_ERR_ARG, "fw_set_sdf: bad argument");
    AssetHost &A = w->assets[asset_id];
    for (int a = 0; a < 3; ++a) { A.lo[a] = lo[a]; A.dims[a] = dims[a]; }
    A.h = h;
    const long long n = (long long)dims[0] * dims[1] * dims[2];
    dfree(A.d_grid);
    CK(cudaMalloc(&A.d_grid, sizeof(float) * n));
    CK(cudaMemcpy(A.d_grid, values, sizeof(float) * n, cudaMemcpyHostToDevice));
    return finish_grid(w, A);
}

fw_status fw_get_sdf(fw_world *w, int asset_id, float lo[3], float *h, int dims[3], float *values) {
    if (!ready(w)) return FW_ERR_ARG;
    if (asset_id < 0 || asset_id >= (int)w->assets.size()) return fail(w, FW_ERR_ARG, "fw_get_sdf: bad asset");
    AssetHost &A = w->assets[asset_id];
    if (!A.has_sdf) return fail(w, FW_ERR_STATE, "fw_get_sdf: asset has no SDF");
    if (lo) for (int a = 0; a < 3; ++a) lo[a] = A.lo[a];
    if (h) *h = A.h;
    if (dims) for (int a = 0; a < 3; ++a) dims[a] = A.dims[a];
    if (values) {
        const long long n = (long long)A.dims[0] * A.dims[1] * A.dims[2];
        CK(cudaMemcpy(values, A.d_grid, sizeof(float) * n, cudaMemcpyDeviceToHost));
    }
    return FW_OK;
}

fw_status fw_add_env_bodies(fw_world *w, int n_envs, const fw_body_desc *bd, int n_per_env, const int *pairs,
                            int n_pairs, int *first_env_out) {
    if (!ready(w)) return FW_ERR_ARG;
    if (n_envs < 1 || !bd || n_per_env < 1 || n_per_env > 8 || n_pairs < 0 || n_pairs > 63 || (n_pairs > 0 && !pairs))
        return fail(w, FW_ERR_ARG, "fw_add_env_bodies: bad sizes (1..8 bodies, 0..63 pairs per env)");
    for (int k = 0; k < n_pairs; ++k) {
        const int a = pairs[2 * k], b = pairs[2 * k + 1];
        if (a < 0 || a >= n_per_env || b < 0 || b >= n_per_env || a == b)
            return fail(w, FW_ERR_ARG, "fw_add_env_bodies: bad pair");
    }
    for (int i = 0; i < n_envs * n_per_env; ++i) {
        const fw_body_desc &d = bd[i];
        if (d.asset < 0 || d.asset >= (int)w->assets.size() || d.type < 0 || d.type > 3)
            return fail(w, FW_ERR_ARG, "fw_add_env_bodies: bad body descriptor");
    }
    for (int e = 0; e < n_envs; ++e)
        for (int k = 0; k < n_pairs; ++k) {
            const AssetHost &Aa = w->assets[bd[e * n_per_env + pairs[2 * k]].asset];
            const AssetHost &Ab = w->assets[bd[e * n_per_env + pairs[2 * k + 1]].asset];
            if (Aa.S.empty() && w->cfg.contact_gen == 0)   // per-triangle generation needs only the mesh
                return fail(w, FW_ERR_STATE, "fw_add_env_bodies: point body has no sample points");
            if (!Ab.has_sdf) return fail(w, FW_ERR_STATE, "fw_add_env_bodies: SDF body has no baked SDF");
        }
    // validate everything before appending anything
    for (int i = 0; i < n_envs * n_per_env; ++i) {
        const fw_body_desc &d = bd[i];
        const double qn = (double)d.quat[0] * d.quat[0] + (double)d.quat[1] * d.quat[1] +
                          (double)d.quat[2] * d.quat[2] + (double)d.quat[3] * d.quat[3];
        const double an = (double)d.axis[0] * d.axis[0] + (double)d.axis[1] * d.axis[1] + (double)d.axis[2] * d.axis[2];
        if (!(qn > 0)) return fail(w, FW_ERR_ARG, "fw_add_env_bodies: zero quaternion");
        if (d.type == FW_BODY_FIXED_AXIS && !(an > 0)) return fail(w, FW_ERR_ARG, "fw_add_env_bodies: zero axis");
        BodyProps P;
        if (!body_props(w, d, P)) return fail(w, FW_ERR_ARG, "fw_add_env_bodies: singular inertia");
    }
    if (w->cfg.solver == 1)
        for (int e = 0; e < n_envs; ++e) {
            int movable = 0;
            for (int i = 0; i < n_per_env; ++i) {
                const int t = bd[e * n_per_env + i].type;
                movable += (t == FW_BODY_DYNAMIC || t == FW_BODY_FIXED_AXIS) ? 1 : 0;
            }
            if (movable > 1)
                return fail(w, FW_ERR_ARG, "fw_add_env_bodies: the Jacobi solver takes envs with one movable body");
        }
    const int e0 = (int)w->envs.size();
    long long scratch = 0, rows = 0;
    for (auto &P : w->pairs) scratch = std::max(scratch, (long long)P.scratch_off + 2LL * pair_sources(w, P.asset_a));
    for (auto &E : w->envs) rows = std::max(rows, (long long)E.row_off + env_row_span(E));
    long long more = 0;
    for (int e = 0; e < n_envs; ++e)
        for (int k = 0; k < n_pairs; ++k) more += 2LL * pair_sources(w, bd[e * n_per_env + pairs[2 * k]].asset);
    if (scratch + more > 0x7FFFFFFFLL) return fail(w, FW_ERR_ARG, "fw_add_env_bodies: too many samples in total");
    if (rows + (long long)n_envs * (2LL * n_pairs * cap_pair(w) + kRowPad) > 0x7FFFFFFFLL)
        return fail(w, FW_ERR_ARG, "fw_add_env_bodies: too many contact rows in total");
    for (int e = 0; e < n_envs; ++e) {
        EnvDev E;
        memset(&E, 0, sizeof E);
        E.first_body = (int)w->props.size();
        E.n_bodies = n_per_env;
        E.first_pair = (int)w->pairs.size();
        E.n_pairs = n_pairs;
        E.row_off = (int)rows;
        E.row_cap = n_pairs * cap_pair(w);
        E.pile = -1;
        E.movable = -1;
        for (int i = 0; i < n_per_env; ++i) {
            const int t = bd[e * n_per_env + i].type;
            if (t == FW_BODY_DYNAMIC || t == FW_BODY_FIXED_AXIS) E.movable = (E.movable == -1) ? i : -2;
        }
        rows += env_row_span(E);
        for (int i = 0; i < n_per_env; ++i) append_body(w, bd[e * n_per_env + i]);
        for (int k = 0; k < n_pairs; ++k) {
            PairDev P;
            memset(&P, 0, sizeof P);
            P.local_a = pairs[2 * k];
            P.local_b = pairs[2 * k + 1];
            P.a = E.first_body + P.local_a;
            P.b = E.first_body + P.local_b;
            P.asset_a = w->props[P.a].asset;
            P.asset_b = w->props[P.b].asset;
            P.env = e0 + e;
            P.mu = (float)std::sqrt((double)w->props[P.a].mu * (double)w->props[P.b].mu);
            P.scratch_off = (int)scratch;
            scratch += 2LL * pair_sources(w, P.asset_a);
            w->pairs.push_back(P);
        }
        w->envs.push_back(E);
        ++w->n_regular;
    }
    w->topo_dirty = true;
    if (first_env_out) *first_env_out = e0;
    return FW_OK;
}

fw_status fw_add_pile(fw_world *w, const fw_body_desc *bd, int n_bodies, int max_pairs, int max_contacts,
                      int *env_out) {
    if (!ready(w)) return FW_ERR_ARG;
    if (!bd || n_bodies < 1 || n_bodies > kMaxPileBodies || max_pairs < 0 || max_contacts < 0)
        return fail(w, FW_ERR_ARG, "fw_add_pile: bad sizes (1..1024 bodies, capacities >= 0)");
    if (w->cfg.contact_gen != 0 || w->cfg.solver != 0)
        return fail(w, FW_ERR_ARG, "fw_add_pile: piles take per-sample contacts and the Gauss-Seidel solver");
    const long long pcap = max_pairs > 0 ? max_pairs : (long long)kPilePairsPerBody * n_bodies;
    const long long rcap = max_contacts > 0 ? max_contacts : (long long)kPileRowsPerBody * n_bodies;
    if (pcap > kPileMaxPairs || rcap >= kPileMaxRows)
        return fail(w, FW_ERR_ARG, "fw_add_pile: capacities too large (65535 pairs, 2^21 - 1 contact rows)");
    if (pile_smem_bytes(n_bodies, (int)pcap) > (size_t)w->pile_optin)
        return fail(w, FW_ERR_ARG, "fw_add_pile: the pile does not fit the solve's shared memory");
    for (int i = 0; i < n_bodies; ++i) {
        const fw_body_desc &d = bd[i];
        if (d.asset < 0 || d.asset >= (int)w->assets.size() || d.type < 0 || d.type > 3)
            return fail(w, FW_ERR_ARG, "fw_add_pile: bad body descriptor");
        const double qn = (double)d.quat[0] * d.quat[0] + (double)d.quat[1] * d.quat[1] +
                          (double)d.quat[2] * d.quat[2] + (double)d.quat[3] * d.quat[3];
        const double an = (double)d.axis[0] * d.axis[0] + (double)d.axis[1] * d.axis[1] + (double)d.axis[2] * d.axis[2];
        if (!(qn > 0)) return fail(w, FW_ERR_ARG, "fw_add_pile: zero quaternion");
        if (d.type == FW_BODY_FIXED_AXIS && !(an > 0)) return fail(w, FW_ERR_ARG, "fw_add_pile: zero axis");
        BodyProps P;
        if (!body_props(w, d, P)) return fail(w, FW_ERR_ARG, "fw_add_pile: singular inertia");
        // a body takes part in pairs through its samples and / or its SDF, whichever it has
        if (d.type != FW_BODY_STATIC && d.type != FW_BODY_KINEMATIC && w->assets[d.asset].S.empty() &&
            !w->assets[d.asset].has_sdf)
            return fail(w, FW_ERR_STATE, "fw_add_pile: a movable body has neither samples nor an SDF");
    }
    EnvDev E;
    memset(&E, 0, sizeof E);
    E.first_body = (int)w->props.size();
    E.n_bodies = n_bodies;
    E.movable = -1;
    E.pile = (int)w->piles.size();
    PileDev P;
    memset(&P, 0, sizeof P);
    P.env = (int)w->envs.size();
    P.first_body = E.first_body;
    P.n_bodies = n_bodies;
    P.pcap = (int)pcap;
    P.rcap = (int)rcap;
    for (int i = 0; i < n_bodies; ++i) append_body(w, bd[i]);
    w->piles.push_back(P);
    w->envs.push_back(E);
    w->topo_dirty = true;
    if (env_out) *env_out = P.env;
    return FW_OK;
}

fw_status fw_step(fw_world *w, int n_substeps, int n_iters) {
    if (!ready(w)) return FW_ERR_ARG;
    if (n_substeps < 1 || n_iters < 0) return fail(w, FW_ERR_ARG, "fw_step: bad substeps/iterations");
    fw_status st = ensure_device(w);
    if (st != FW_OK) return st;
    const float hs = w->cfg.dt / (float)n_substeps;
    if (w->timing) return enqueue_substeps(w, w->stream, n_substeps, hs, n_iters, true, true);
    if (!w->gexec || w->g_sub != n_substeps || w->g_iters != n_iters) {
        drop_graph(w);
        CK(cudaStreamBeginCapture(w->cap_stream, cudaStreamCaptureModeThreadLocal));
        const fw_status s2 = enqueue_substeps(w, w->cap_stream, n_substeps, hs, n_iters, true, false);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(w->cap_stream, &g);
        if (s2 != FW_OK) { if (g) cudaGraphDestroy(g); return s2; }
        if (e != cudaSuccess) return cuda_fail(w, e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&w->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { w->gexec = nullptr; return cuda_fail(w, e, "cudaGraphInstantiate"); }
        w->g_sub = n_substeps;
        w->g_iters = n_iters;
    }
    CK(cudaGraphLaunch(w->gexec, w->stream));
    return FW_OK;
}

fw_status fw_substep(fw_world *w, float hs, int n_iters, int detect) {
    if (!ready(w)) return FW_ERR_ARG;
    if (!(hs > 0) || n_iters < 0) return fail(w, FW_ERR_ARG, "fw_substep: bad arguments");
    fw_status st = ensure_device(w);
    if (st != FW_OK) return st;
    return enqueue_substeps(w, w->stream, 1, hs, n_iters, detect != 0, false);
}

fw_status fw_collide(fw_world *w) {
    if (!ready(w)) return FW_ERR_ARG;
    fw_status st = ensure_device(w);
    if (st != FW_OK) return st;
    const SimParams p = sim_params(w, w->cfg.dt, 0);
    if (w->n_regular > 0) CK(launch_detect(p, w->stream));
    if (!w->piles.empty()) {
        const SimParams q = pile_params(w, w->cfg.dt, 0);
        st = enqueue_pile_detect(w, q, w->stream);
        if (st != FW_OK) return st;
        CK(launch_reduce(q, w->stream));
    }
    return FW_OK;
}

fw_status fw_get_contacts(fw_world *w, int env, fw_contact *out, int cap, int *n_out) {
    if (!ready(w)) return FW_ERR_ARG;
    if (env < 0 || env >= (int)w->envs.size() || (cap > 0 && !out) || !n_out)
        return fail(w, FW_ERR_ARG, "fw_get_contacts: bad argument");
    fw_status st = ensure_device(w);
    if (st != FW_OK) return st;
    const EnvDev &E = w->envs[env];
    const int cp = cap_pair(w);
    // the env's pairs: its listed pairs, or its pile's current pairs
    int n_pairs = E.n_pairs;
    const int *d_counts = w->d_counts + E.first_pair;
    const DContact *d_con = w->d_contacts + (size_t)E.first_pair * cp;
    if (E.pile >= 0) {
        if ((st = pile_pair_count(w, E.pile, &n_pairs)) != FW_OK) return st;
        d_counts = w->d_pccounts + (size_t)E.pile * w->pile_pcap;
        d_con = w->d_pcontacts + (size_t)E.pile * w->pile_pcap * cp;
    }
    std::vector<int> counts(n_pairs);
    if (n_pairs > 0)
        CK(cudaMemcpyAsync(counts.data(), d_counts, sizeof(int) * n_pairs, cudaMemcpyDeviceToHost, w->stream));
    std::vector<DContact> dc((size_t)n_pairs * cp);
    if (n_pairs > 0)
        CK(cudaMemcpyAsync(dc.data(), d_con, sizeof(DContact) * dc.size(), cudaMemcpyDeviceToHost, w->stream));
    CK(cudaStreamSynchronize(w->stream));
    int n = 0;
    for (int k = 0; k < n_pairs; ++k)
        for (int i = 0; i < std::min(counts[k], cp); ++i, ++n) {
            if (n >= cap) continue;
            const DContact &c = dc[(size_t)k * cp + i];
            fw_contact &o = out[n];
            o.sample = c.sample_patch & 0xFFFFFF;
            o.patch = (int)((unsigned)c.sample_patch >> 24);
            o.pair = k;
            o.phi = c.phi;
            for (int a = 0; a < 3; ++a) {
                o.xa[a] = c.xa[a];
                o.n[a] = c.n[a];
                o.xb[a] = c.xa[a] - c.phi * c.n[a];
            }
        }
    *n_out = n;
    st = check_status(w);
    if (st != FW_OK) return st;
    return n > cap ? fail(w, FW_ERR_OVERFLOW, "fw_get_contacts: cap too small") : FW_OK;
}

fw_status fw_set_contacts(fw_world *w, int env, const fw_contact *in, int n) {
    if (!ready(w)) return FW_ERR_ARG;
    if (env < 0 || env >= (int)w->envs.size() || n < 0 || (n > 0 && !in))
        return fail(w, FW_ERR_ARG, "fw_set_contacts: bad argument");
    fw_status st = ensure_device(w);
    if (st != FW_OK) return st;
    const EnvDev &E = w->envs[env];
    const int cp = cap_pair(w);
    int n_pairs = E.n_pairs;
    int *d_counts = w->d_counts + E.first_pair;
    DContact *d_con = w->d_contacts + (size_t)E.first_pair * cp;
    if (E.pile >= 0) {   // the pile's pairs of its last detection keep their order
        if ((st = pile_pair_count(w, E.pile, &n_pairs)) != FW_OK) return st;
        d_counts = w->d_pccounts + (size_t)E.pile * w->pile_pcap;
        d_con = w->d_pcontacts + (size_t)E.pile * w->pile_pcap * cp;
    }
    std::vector<int> counts(n_pairs, 0);
    std::vector<DContact> dc((size_t)n_pairs * cp);
    int last_pair = 0;
    for (int i = 0; i < n; ++i) {
        const int k = in[i].pair;
        if (k < 0 || k >= n_pairs || k < last_pair)
            return fail(w, FW_ERR_ARG, "fw_set_contacts: pairs must be grouped in order");
        last_pair = k;
        if (counts[k] >= cp) return fail(w, FW_ERR_OVERFLOW, "fw_set_contacts: too many contacts for a pair");
        DContact &c = dc[(size_t)k * cp + counts[k]++];
        for (int a = 0; a < 3; ++a) { c.xa[a] = in[i].xa[a]; c.n[a] = in[i].n[a]; }
        c.phi = in[i].phi;
        c.sample_patch = (in[i].sample & 0xFFFFFF) | ((in[i].patch & 0xFF) << 24);
    }
    if (n_pairs > 0) {
        CK(cudaMemcpyAsync(d_counts, counts.data(), sizeof(int) * n_pairs, cudaMemcpyHostToDevice, w->stream));
        CK(cudaMemcpyAsync(d_con, dc.data(), sizeof(DContact) * dc.size(), cudaMemcpyHostToDevice, w->stream));
    }
    CK(cudaStreamSynchronize(w->stream));
    return FW_OK;
}

fw_status fw_get_state(fw_world *w, float *pos, float *quat, float *linvel, float *angvel, int device_ptrs) {
    if (!ready(w)) return FW_ERR_ARG;
    fw_status st = ensure_device(w);
    if (st != FW_OK) return st;
    const size_t nb = w->props.size();
    const cudaMemcpyKind k = device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (pos) CK(cudaMemcpyAsync(pos, w->d_pos, sizeof(float) * 3 * nb, k, w->stream));
    if (quat) CK(cudaMemcpyAsync(quat, w->d_quat, sizeof(float) * 4 * nb, k, w->stream));
    if (linvel) CK(cudaMemcpyAsync(linvel, w->d_vel, sizeof(float) * 3 * nb, k, w->stream));
    if (angvel) CK(cudaMemcpyAsync(angvel, w->d_ang, sizeof(float) * 3 * nb, k, w->stream));
    if (!device_ptrs) {
        CK(cudaStreamSynchronize(w->stream));
        return check_status(w);
    }
    return FW_OK;
}

fw_status fw_set_state(fw_world *w, const float *pos, const float *quat, const float *linvel, const float *angvel,
                       int device_ptrs) {
    if (!ready(w)) return FW_ERR_ARG;
    fw_status st = ensure_device(w);
    if (st != FW_OK) return st;
    const size_t nb = w->props.size();
    const cudaMemcpyKind k = device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (pos) CK(cudaMemcpyAsync(w->d_pos, pos, sizeof(float) * 3 * nb, k, w->stream));
    if (quat) {
        CK(cudaMemcpyAsync(w->d_quat, quat, sizeof(float) * 4 * nb, k, w->stream));
        CK(launch_normalize_quats(w->d_quat, (int)nb, w->stream));
    }
    if (linvel) CK(cudaMemcpyAsync(w->d_vel, linvel, sizeof(float) * 3 * nb, k, w->stream));
    if (angvel) CK(cudaMemcpyAsync(w->d_ang, angvel, sizeof(float) * 3 * nb, k, w->stream));
    if (!device_ptrs) CK(cudaStreamSynchronize(w->stream));   // host buffers may be reused at return
    return FW_OK;
}

fw_status fw_query_sdf(fw_world *w, int asset_id, const float *pts, int n, float *phi, float *grad, int device_ptrs) {
    if (!ready(w)) return FW_ERR_ARG;
    if (asset_id < 0 || asset_id >= (int)w->assets.size() || n < 0 || (n > 0 && (!pts || !phi || !grad)))
        return fail(w, FW_ERR_ARG, "fw_query_sdf: bad argument");
    AssetHost &A = w->assets[asset_id];
    if (!A.has_sdf) return fail(w, FW_ERR_STATE, "fw_query_sdf: asset has no SDF");
    if (n == 0) return FW_OK;
    const AssetDev g = asset_view(A, w->cfg.sdf_fp16 != 0);
    if (device_ptrs) {
        CK(launch_query_sdf(g, pts, n, phi, grad, w->stream));
        return FW_OK;
    }
    float *d = nullptr;
    CK(cudaMalloc(&d, sizeof(float) * 7 * (size_t)n));
    CK(cudaMemcpyAsync(d, pts, sizeof(float) * 3 * (size_t)n, cudaMemcpyHostToDevice, w->stream));
    CK(launch_query_sdf(g, d, n, d + 3 * (size_t)n, d + 4 * (size_t)n, w->stream));
    CK(cudaMemcpyAsync(phi, d + 3 * (size_t)n, sizeof(float) * n, cudaMemcpyDeviceToHost, w->stream));
    CK(cudaMemcpyAsync(grad, d + 4 * (size_t)n, sizeof(float) * 3 * (size_t)n, cudaMemcpyDeviceToHost, w->stream));
    CK(cudaStreamSynchronize(w->stream));
    cudaFree(d);
    return FW_OK;
}

fw_status fw_query_pair(fw_world *w, int env, int pair, float *phi, float *normal, int device_ptrs) {
    if (!ready(w)) return FW_ERR_ARG;
    if (env < 0 || env >= (int)w->envs.size() || pair < 0 || pair >= w->envs[env].n_pairs || !phi || !normal)
        return fail(w, FW_ERR_ARG, "fw_query_pair: bad argument");
    fw_status st = ensure_device(w);
    if (st != FW_OK) return st;
    const int pi = w->envs[env].first_pair + pair;
    const int ns = (int)(w->assets[w->pairs[pi].asset_a].S.size() / 3);
    const SimParams p = sim_params(w, w->cfg.dt, 0);
    if (device_ptrs) {
        CK(launch_query_pair(p, pi, phi, normal, w->stream, ns));
        return FW_OK;
    }
    float *d = nullptr;
    CK(cudaMalloc(&d, sizeof(float) * 4 * (size_t)ns));
    CK(launch_query_pair(p, pi, d, d + ns, w->stream, ns));
    CK(cudaMemcpyAsync(phi, d, sizeof(float) * ns, cudaMemcpyDeviceToHost, w->stream));
    CK(cudaMemcpyAsync(normal, d + ns, sizeof(float) * 3 * (size_t)ns, cudaMemcpyDeviceToHost, w->stream));
    CK(cudaStreamSynchronize(w->stream));
    cudaFree(d);
    return FW_OK;
}

fw_status fw_tri_contacts(fw_world *w, int env, int pair, float *x, float *phi, float *normal, int device_ptrs) {
    if (!ready(w)) return FW_ERR_ARG;
    if (env < 0 || env >= (int)w->envs.size() || pair < 0 || pair >= w->envs[env].n_pairs || !x || !phi || !normal)
        return fail(w, FW_ERR_ARG, "fw_tri_contacts: bad argument");
    fw_status st = ensure_device(w);
    if (st != FW_OK) return st;
    const int pi = w->envs[env].first_pair + pair;
    const int nt = (int)(w->assets[w->pairs[pi].asset_a].T.size() / 3);
    const SimParams p = sim_params(w, w->cfg.dt, 0);
    if (device_ptrs) {
        CK(launch_tri_pair(p, pi, x, phi, normal, w->stream, nt));
        return FW_OK;
    }
    float *d = nullptr;
    CK(cudaMalloc(&d, sizeof(float) * 7 * (size_t)nt));
    CK(launch_tri_pair(p, pi, d, d + 3 * (size_t)nt, d + 4 * (size_t)nt, w->stream, nt));
    CK(cudaMemcpyAsync(x, d, sizeof(float) * 3 * (size_t)nt, cudaMemcpyDeviceToHost, w->stream));
    CK(cudaMemcpyAsync(phi, d + 3 * (size_t)nt, sizeof(float) * nt, cudaMemcpyDeviceToHost, w->stream));
    CK(cudaMemcpyAsync(normal, d + 4 * (size_t)nt, sizeof(float) * 3 * (size_t)nt, cudaMemcpyDeviceToHost, w->stream));
    CK(cudaStreamSynchronize(w->stream));
    cudaFree(d);
    return FW_OK;
}

fw_status fw_reduce(fw_world *w, const fw_candidate *cands, int n, fw_contact *out, int cap, int *n_out,
                    int *n_patches) {
    if (!ready(w)) return FW_ERR_ARG;
    if (n < 0 || (n > 0 && !cands) || !n_out || (cap > 0 && !out)) return fail(w, FW_ERR_ARG, "fw_reduce: bad argument");
    std::vector<fw_candidate> c(cands, cands + n);
    std::stable_sort(c.begin(), c.end(), [](const fw_candidate &a, const fw_candidate &b) { return a.sample < b.sample; });
    int max_s = -1;
    for (int i = 0; i < n; ++i) {
        if (c[i].sample < 0 || c[i].sample >= (1 << 24)) return fail(w, FW_ERR_ARG, "fw_reduce: sample out of range");
        if (i > 0 && c[i].sample == c[i - 1].sample) return fail(w, FW_ERR_ARG, "fw_reduce: duplicate sample");
        max_s = std::max(max_s, c[i].sample);
    }
    const int cp = cap_pair(w);
    float *d_c = nullptr;
    float4 *d_scr = nullptr;
    DContact *d_out = nullptr;
    int *d_cnt = nullptr;
    CK(cudaMalloc(&d_c, sizeof(fw_candidate) * std::max(n, 1)));
    CK(cudaMalloc(&d_scr, sizeof(float4) * 2 * (size_t)(max_s + 2)));
    CK(cudaMalloc(&d_out, sizeof(DContact) * cp));
    CK(cudaMalloc(&d_cnt, sizeof(int) * 2));
    if (n > 0) CK(cudaMemcpy(d_c, c.data(), sizeof(fw_candidate) * n, cudaMemcpyHostToDevice));
    CK(cudaMemsetAsync(d_cnt, 0, sizeof(int) * 2, w->stream));
    SimParams p = sim_params(w, w->cfg.dt, 0);
    p.scratch = d_scr;
    CK(launch_reduce_list(p, d_c, n, d_out, d_cnt, d_cnt + 1, w->stream));
    int hc[2];
    std::vector<DContact> h(cp);
    CK(cudaMemcpyAsync(hc, d_cnt, sizeof(int) * 2, cudaMemcpyDeviceToHost, w->stream));
    CK(cudaMemcpyAsync(h.data(), d_out, sizeof(DContact) * cp, cudaMemcpyDeviceToHost, w->stream));
    CK(cudaStreamSynchronize(w->stream));
    cudaFree(d_c); cudaFree(d_scr); cudaFree(d_out); cudaFree(d_cnt);
    const int k = hc[0];
    for (int i = 0; i < k && i < cap; ++i) {
        fw_contact &o = out[i];
        o.sample = h[i].sample_patch & 0xFFFFFF;
        o.patch = (int)((unsigned)h[i].sample_patch >> 24);
        o.pair = 0;
        o.phi = h[i].phi;
        for (int a = 0; a < 3; ++a) {
            o.xa[a] = h[i].xa[a];
            o.n[a] = h[i].n[a];
            o.xb[a] = h[i].xa[a] - h[i].phi * h[i].n[a];
        }
    }
    *n_out = k;
    if (n_patches) *n_patches = hc[1];
    const fw_status st = check_status(w);
    if (st != FW_OK) return st;
    return k > cap ? fail(w, FW_ERR_OVERFLOW, "fw_reduce: cap too small") : FW_OK;
}

fw_status fw_reduce_noalloc(fw_world *w, const fw_candidate *d_cands, int n, fw_contact *d_out, int cap,
                            int *d_counts) {
    if (!ready(w)) return FW_ERR_ARG;
    if (n < 0 || cap < 0 || !d_counts || (n > 0 && !d_cands) || (cap > 0 && !d_out))
        return fail(w, FW_ERR_ARG, "fw_reduce_noalloc: bad argument");
    if (n > kNoAllocMaxSamples)
        return fail(w, FW_ERR_ARG, "fw_reduce_noalloc: more than 65536 candidates (its fixed scratch holds "
                                   "sample ids 0..65535)");
    const SimParams p = sim_params(w, w->cfg.dt, 0);
    CK(launch_reduce_noalloc(p, w->cfg.device, reinterpret_cast<const float *>(d_cands), n, d_out, cap, d_counts,
                             w->stream));
    return FW_OK;
}

fw_status fw_sync(fw_world *w) {
    if (!ready(w)) return FW_ERR_ARG;
    CK(cudaStreamSynchronize(w->stream));
    return check_status(w);
}

fw_status fw_set_timing(fw_world *w, int enable) {
    if (!w) return FW_ERR_ARG;
    w->timing = enable != 0;
    return FW_OK;
}

fw_status fw_get_timings(fw_world *w, float *ms, int n) {
    if (!ready(w) || !ms || n < 4) return fail(w, FW_ERR_ARG, "fw_get_timings: need 4 outputs");
    CK(cudaStreamSynchronize(w->stream));
    double qry = 0, red = 0, sol = 0;
    int nd = 0, ns = 0;
    for (size_t i = 0; i + 3 < w->ev_used.size(); i += 4) {
        float a = 0, b = 0, c = 0;
        CK(cudaEventElapsedTime(&a, w->ev_used[i], w->ev_used[i + 1]));
        CK(cudaEventElapsedTime(&b, w->ev_used[i + 1], w->ev_used[i + 2]));
        CK(cudaEventElapsedTime(&c, w->ev_used[i + 2], w->ev_used[i + 3]));
        qry += a;
        red += b;
        sol += c;
        ++nd;
        ++ns;
    }
    for (auto e : w->ev_used) w->ev_pool.push_back(e);
    w->ev_used.clear();
    ms[0] = (float)(qry + red); ms[1] = (float)sol; ms[2] = (float)nd; ms[3] = (float)ns;
    if (n > 4) ms[4] = (float)qry;
    if (n > 5) ms[5] = (float)red;
    for (int i = 6; i < n; ++i) ms[i] = 0.f;
    return FW_OK;
}

fw_status fw_set_solve_shape(fw_world *w, int envs_per_warp, int warps_per_block) {
    if (!w) return FW_ERR_ARG;
    if (!(envs_per_warp == 0 || envs_per_warp == 1 || envs_per_warp == 2 || envs_per_warp == 4 || envs_per_warp == 8) ||
        warps_per_block < 0 || warps_per_block > kSolveMaxWarps)
        return fail(w, FW_ERR_ARG, "fw_set_solve_shape: envs_per_warp in {0,1,2,4,8}, warps_per_block in 0..4");
    if (w->solve_groups != envs_per_warp || w->solve_warps != warps_per_block) drop_graph(w);
    w->solve_groups = envs_per_warp;
    w->solve_warps = warps_per_block;
    return FW_OK;
}

fw_status fw_autotune_solve(fw_world *w, int n_substeps, int n_iters, int trials, int *envs_per_warp,
                            int *warps_per_block, float *best_ms) {
    if (!ready(w)) return FW_ERR_ARG;
    if (n_substeps < 1 || n_iters < 0 || trials < 1) return fail(w, FW_ERR_ARG, "fw_autotune_solve: bad arguments");
    fw_status st = ensure_device(w);
    if (st != FW_OK) return st;
    const int nb = (int)w->props.size();
    if (nb == 0 || w->n_regular == 0) return FW_OK;   // the shape is that of the per-env solve
    // the state is saved and put back around every candidate, so tuning does not advance it
    float *save = nullptr;
    CK(cudaMalloc(&save, sizeof(float) * 13 * nb));
    float *const src[4] = {w->d_pos, w->d_quat, w->d_vel, w->d_ang};
    const size_t len[4] = {3, 4, 3, 3};
    auto copy_state = [&](bool to_save) -> cudaError_t {
        size_t off = 0;
        for (int k = 0; k < 4; ++k) {
            const size_t bytes = sizeof(float) * len[k] * nb;
            cudaError_t e = to_save ? cudaMemcpyAsync(save + off, src[k], bytes, cudaMemcpyDeviceToDevice, w->stream)
                                    : cudaMemcpyAsync(src[k], save + off, bytes, cudaMemcpyDeviceToDevice, w->stream);
            if (e != cudaSuccess) return e;
            off += len[k] * nb;
        }
        return cudaSuccess;
    };
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = copy_state(true);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    SimParams p = sim_params(w, w->cfg.dt / (float)n_substeps, n_iters);
    if (e == cudaSuccess) e = launch_detect(p, w->stream);   // contacts of the current state
    // Shared memory per env: room for twice the largest row count seen now (a power of two,
    // at least 64 rows) when that is below the envs' row capacity.  Fewer bytes per env let
    // more envs run at once; an env that later outgrows it keeps its impulses in global
    // memory (same update, slower).
    if (e == cudaSuccess) {
        std::vector<int> cnt(w->pairs.size());
        e = cudaMemcpyAsync(cnt.data(), w->d_counts, sizeof(int) * cnt.size(), cudaMemcpyDeviceToHost, w->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
        if (e == cudaSuccess) {
            const int cp = cap_pair(w);
            int max_nr = 0, rc = 0;
            for (const auto &E : w->envs) {
                int nr = 0;
                for (int k = 0; k < E.n_pairs; ++k) nr += std::min(cnt[E.first_pair + k], cp);
                max_nr = std::max(max_nr, nr);
                rc = std::max(rc, E.row_cap);
            }
            int lam = 64;
            while (lam < 2 * max_nr) lam *= 2;
            const int rows = lam < rc ? lam : 0;
            if (rows != w->lam_rows) { w->lam_rows = rows; drop_graph(w); }
            p = sim_params(w, w->cfg.dt / (float)n_substeps, n_iters);
        }
    }
    int bg = 0, bw = 0;
    float best = 1e30f;
    const int gs[4] = {1, 2, 4, 8};
    for (int gi = 0; gi < 4 && e == cudaSuccess; ++gi)
        for (int wp = 1; wp <= kSolveMaxWarps && e == cudaSuccess; ++wp) {
            const SolveShape sh = solve_shape(p.n_envs, p.lam_cap, gs[gi], wp, w->max_dyn_smem, w->n_sm);
            if (sh.groups != gs[gi] || sh.warps != wp) continue;   // does not fit: lowered to another candidate
            e = copy_state(false);
            if (e == cudaSuccess) e = launch_solve(p, sh, w->stream);   // warm
            if (e == cudaSuccess) e = copy_state(false);
            if (e == cudaSuccess) e = cudaEventRecord(a, w->stream);
            for (int t = 0; t < trials && e == cudaSuccess; ++t) e = launch_solve(p, sh, w->stream);
            if (e == cudaSuccess) e = cudaEventRecord(b, w->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(b);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
            ms /= (float)trials;
            // a later shape must win by more than 1% (timing noise would otherwise flip
            // between shapes of equal speed from run to run)
            if (e == cudaSuccess && ms < best * 0.99f) { best = ms; bg = gs[gi]; bw = wp; }
        }
    if (e == cudaSuccess) e = copy_state(false);
    if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(save);
    if (e != cudaSuccess) return cuda_fail(w, e, "fw_autotune_solve");
    if (bg > 0) {
        if (w->solve_groups != bg || w->solve_warps != bw) drop_graph(w);
        w->solve_groups = bg;
        w->solve_warps = bw;
    }
    if (envs_per_warp) *envs_per_warp = bg;
    if (warps_per_block) *warps_per_block = bw;
    if (best_ms) *best_ms = best;
    return FW_OK;
}

fw_status fw_test_stall(fw_world *w, int what) {
    if (!w) return FW_ERR_ARG;
    if (what < 0 || what > 2) return fail(w, FW_ERR_ARG, "fw_test_stall: 0, 1 or 2");
    if (w->stall != what) drop_graph(w);
    w->stall = what;
    return FW_OK;
}

fw_status fw_set_query_cull(fw_world *w, int on) {
    if (!w) return FW_ERR_ARG;
    if (on != 0 && on != 1) return fail(w, FW_ERR_ARG, "fw_set_query_cull: 0 or 1");
    if (w->no_cull != !on) drop_graph(w);
    w->no_cull = !on;
    return FW_OK;
}

fw_status fw_get_query_cull(fw_world *w, int *on) {
    if (!w || !on) return FW_ERR_ARG;
    *on = w->no_cull ? 0 : 1;
    return FW_OK;
}

fw_status fw_set_detect_shape(fw_world *w, int query_threads, int reduce_warps) {
    if (!w) return FW_ERR_ARG;
    if (!(query_threads == 0 || query_threads == 128 || query_threads == 256 || query_threads == 512) ||
        !(reduce_warps == 0 || reduce_warps == 2 || reduce_warps == 4 || reduce_warps == 8))
        return fail(w, FW_ERR_ARG, "fw_set_detect_shape: query_threads in {0,128,256,512}, reduce_warps in {0,2,4,8}");
    if (w->query_threads != query_threads || w->reduce_warps != reduce_warps) drop_graph(w);
    w->query_threads = query_threads;
    w->reduce_warps = reduce_warps;
    return FW_OK;
}

fw_status fw_get_detect_shape(fw_world *w, int *query_threads, int *reduce_warps) {
    if (!w) return FW_ERR_ARG;
    if (query_threads) *query_threads = w->query_threads > 0 ? w->query_threads : 256;
    if (reduce_warps) *reduce_warps = w->reduce_warps > 0 ? w->reduce_warps : 4;
    return FW_OK;
}

fw_status fw_autotune_detect(fw_world *w, int trials, int *query_threads, int *reduce_warps, float *best_ms) {
    if (!ready(w)) return FW_ERR_ARG;
    if (trials < 1) return fail(w, FW_ERR_ARG, "fw_autotune_detect: trials >= 1");
    fw_status st = ensure_device(w);
    if (st != FW_OK) return st;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const bool piles = !w->piles.empty();
    // one detection pass (query of every work item, then the reduction of every pair) for
    // the given shape; the reduction reads only the query's output, so it is timed alone
    auto time_phase = [&](int qt, int rw, bool query, float *ms) -> fw_status {
        w->query_threads = qt;
        w->reduce_warps = rw;
        SimParams p = sim_params(w, w->cfg.dt, 0);
        const SimParams q = piles ? pile_params(w, w->cfg.dt, 0) : p;
        // one untimed pass first: a kernel's first launch also loads its module
        for (int t = -1; t < trials; ++t) {
            if (t == 0) CK(cudaEventRecord(e0, w->stream));
            if (query) {
                if (w->n_regular > 0) CK(launch_query(p, w->stream));
                if (piles) CK(launch_query(q, w->stream));
            } else {
                if (w->n_regular > 0) CK(launch_reduce(p, w->stream));
                if (piles) CK(launch_reduce(q, w->stream));
            }
        }
        CK(cudaEventRecord(e1, w->stream));
        CK(cudaEventSynchronize(e1));
        CK(cudaEventElapsedTime(ms, e0, e1));
        *ms /= (float)trials;
        return FW_OK;
    };
    // the pile pair lists (if any) and every query's output at the current poses
    st = fw_collide(w);
    int best_q = 256, best_r = 4;
    float bq = 1e30f, br = 1e30f;
    for (int qt : {256, 128, 512}) {   // the query with the default reduction
        float ms = 0.f;
        if (st == FW_OK) st = time_phase(qt, 4, true, &ms);
        if (st == FW_OK && ms < bq * 0.99f) { bq = ms; best_q = qt; }   // the default first; 1% to beat it
    }
    // the cull (fw_set_query_cull) with the chosen query: kept only where it makes the query
    // more than 10% faster.  Its cost (the groups' tests) is fixed while what it saves can
    // shrink as the bodies come together (a nut running down its bolt: a 3% gain at tuning
    // time was a 7% loss a few frames later); where the geometry keeps most groups out of
    // reach (gear teeth away from the mesh zone) it saves far more than that.
    bool cull = true;
    {
        const int keep = w->no_cull;
        float on_ms = 0.f, off_ms = 0.f;
        w->no_cull = 0;
        if (st == FW_OK) st = time_phase(best_q, 4, true, &on_ms);
        w->no_cull = 1;
        if (st == FW_OK) st = time_phase(best_q, 4, true, &off_ms);
        cull = st == FW_OK && on_ms < off_ms * 0.90f;
        w->no_cull = st == FW_OK ? (cull ? 0 : 1) : keep;
    }
    if (st == FW_OK) st = time_phase(best_q, 4, true, &bq);   // leave the best query's output
    for (int rw : {4, 2, 8}) {
        float ms = 0.f;
        if (st == FW_OK) st = time_phase(best_q, rw, false, &ms);
        if (st == FW_OK && ms < br * 0.99f) { br = ms; best_r = rw; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != FW_OK) return st;
    w->query_threads = best_q;
    w->reduce_warps = best_r;
    // the contacts of the chosen shape (every shape gives the same ones)
    if (w->n_regular > 0) CK(launch_reduce(sim_params(w, w->cfg.dt, 0), w->stream));
    if (piles) CK(launch_reduce(pile_params(w, w->cfg.dt, 0), w->stream));
    drop_graph(w);
    if (query_threads) *query_threads = best_q;
    if (reduce_warps) *reduce_warps = best_r;
    if (best_ms) *best_ms = bq + br;
    return check_status(w);
}

fw_status fw_get_solve_shape(fw_world *w, int *envs_per_warp, int *warps_per_block) {
    if (!w) return FW_ERR_ARG;
    const SimParams p = sim_params(w, 1.0f, 1);
    const SolveShape sh = current_solve_shape(w, p);
    if (envs_per_warp) *envs_per_warp = sh.groups;
    if (warps_per_block) *warps_per_block = sh.warps;
    return FW_OK;
}

fw_status fw_set_body_params(fw_world *w, const float *mass, const float *mu) {
    if (!ready(w)) return FW_ERR_ARG;
    CK(cudaStreamSynchronize(w->stream));
    const int nb = (int)w->props.size(), np = (int)w->pairs.size();
    if (mass)
        for (int i = 0; i < nb; ++i) {
            if (!(mass[i] > 0.0f)) continue;
            BodyProps &P = w->props[i];
            if (!(P.mass > 0.0f)) return fail(w, FW_ERR_ARG, "fw_set_body_params: body has no mass to rescale");
            const float sc = mass[i] / P.mass;
            for (int k = 0; k < 6; ++k) { P.Ib[k] *= sc; P.Ib_inv[k] /= sc; }
            P.mass = mass[i];
            if (P.type == FW_BODY_DYNAMIC) P.invm = 1.0f / mass[i];
        }
    if (mu)
        for (int i = 0; i < np; ++i)
            if (mu[i] >= 0.0f) w->pairs[i].mu = mu[i];
    if (w->d_props && nb > 0) CK(cudaMemcpy(w->d_props, w->props.data(), sizeof(BodyProps) * nb, cudaMemcpyHostToDevice));
    if (w->d_pairs && np > 0) CK(cudaMemcpy(w->d_pairs, w->pairs.data(), sizeof(PairDev) * np, cudaMemcpyHostToDevice));
    return FW_OK;
}

fw_status fw_record_rollout(fw_world *w, int n_substeps, int n_iters) {
    if (!ready(w)) return FW_ERR_ARG;
    if (n_substeps < 1 || n_iters < 0) return fail(w, FW_ERR_ARG, "fw_record_rollout: bad substeps/iterations");
    if (w->cfg.n_vel_iters != 0) return fail(w, FW_ERR_ARG, "fw_record_rollout: needs n_vel_iters = 0");
    if (w->cfg.solver != 0) return fail(w, FW_ERR_ARG, "fw_record_rollout: needs the Gauss-Seidel solver");
    // the tape rebuilds a contact from its surface sample; per-triangle contacts have none
    if (w->cfg.contact_gen != 0)
        return fail(w, FW_ERR_ARG, "fw_record_rollout: needs contact_gen = 0 (per-sample contacts)");
    fw_status st = ensure_device(w);
    if (st != FW_OK) return st;
    std::vector<int> dyn;
    if ((st = diff_envs(w, dyn)) != FW_OK) return st;
    if ((st = diff_alloc(w, n_substeps, n_iters)) != FW_OK) return st;
    if (!dyn.empty()) {
        CK(cudaMemcpyAsync(w->diff.dyn, dyn.data(), sizeof(int) * dyn.size(), cudaMemcpyHostToDevice, w->stream));
        CK(cudaStreamSynchronize(w->stream));   // dyn is a local vector
    }
    const SimParams p = sim_params(w, w->diff.hs, n_iters);
    const int nb = (int)w->props.size();
    for (int si = 0; si < n_substeps; ++si) {
        CK(launch_detect(p, w->stream));
        CK(launch_diff_forward(p, w->diff, si, nb, false, w->stream));
    }
    w->diff_valid = true;
    return FW_OK;
}

fw_status fw_replay_rollout(fw_world *w) {
    if (!ready(w)) return FW_ERR_ARG;
    if (!w->diff_valid) return fail(w, FW_ERR_STATE, "fw_replay_rollout: no recorded rollout");
    fw_status st = ensure_device(w);
    if (st != FW_OK) return st;
    const SimParams p = sim_params(w, w->diff.hs, w->diff.K);
    for (int si = 0; si < w->diff.S; ++si) CK(launch_diff_forward(p, w->diff, si, (int)w->props.size(), true, w->stream));
    return FW_OK;
}

fw_status fw_adjoint_rollout(fw_world *w, const float *g_pos, const float *g_quat, const float *g_linvel,
                             const float *g_angvel, float *d_pos, float *d_quat, float *d_linvel, float *d_angvel,
                             float *d_mass, float *d_mu, int device_ptrs) {
    if (!ready(w)) return FW_ERR_ARG;
    if (!w->diff_valid) return fail(w, FW_ERR_STATE, "fw_adjoint_rollout: no recorded rollout");
    if (!g_pos || !g_quat || !g_linvel || !g_angvel || !d_pos || !d_quat || !d_linvel || !d_angvel || !d_mass || !d_mu)
        return fail(w, FW_ERR_ARG, "fw_adjoint_rollout: NULL pointer");
    const int nb = (int)w->props.size(), np = (int)w->pairs.size();
    const cudaMemcpyKind in_kind = device_ptrs ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
    std::vector<float> g(4 * 13 * (size_t)nb), xb(13 * (size_t)nb);
    float *gp = g.data(), *gq = gp + 3 * nb, *gv = gq + 4 * nb, *gw = gv + 3 * nb;
    CK(cudaStreamSynchronize(w->stream));
    CK(cudaMemcpy(gp, g_pos, sizeof(float) * 3 * nb, in_kind));
    CK(cudaMemcpy(gq, g_quat, sizeof(float) * 4 * nb, in_kind));
    CK(cudaMemcpy(gv, g_linvel, sizeof(float) * 3 * nb, in_kind));
    CK(cudaMemcpy(gw, g_angvel, sizeof(float) * 3 * nb, in_kind));
    for (int i = 0; i < nb; ++i) {
        for (int k = 0; k < 3; ++k) { xb[13 * i + k] = gp[3 * i + k]; xb[13 * i + 7 + k] = gv[3 * i + k]; xb[13 * i + 10 + k] = gw[3 * i + k]; }
        for (int k = 0; k < 4; ++k) xb[13 * i + 3 + k] = gq[4 * i + k];
    }
    DiffState &d = w->diff;
    // everything in stream order on the world's stream (it does not synchronise with the
    // legacy default stream), then one wait before reading back
    CK(cudaMemcpyAsync(d.xb, xb.data(), sizeof(float) * 13 * nb, cudaMemcpyHostToDevice, w->stream));
    CK(cudaMemsetAsync(d.mass_b, 0, sizeof(float) * nb, w->stream));
    CK(cudaMemsetAsync(d.mu_b, 0, sizeof(float) * std::max(np, 1), w->stream));
    const SimParams p = sim_params(w, d.hs, d.K);
    for (int si = d.S - 1; si >= 0; --si) CK(launch_diff_reverse(p, d, si, nb, w->stream));
    CK(cudaStreamSynchronize(w->stream));
    std::vector<float> mb(nb), mub(std::max(np, 1));
    CK(cudaMemcpy(xb.data(), d.xb, sizeof(float) * 13 * nb, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(mb.data(), d.mass_b, sizeof(float) * nb, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(mub.data(), d.mu_b, sizeof(float) * np, cudaMemcpyDeviceToHost));
    std::vector<float> out(13 * (size_t)nb, 0.0f);
    float *op = out.data(), *oq = op + 3 * nb, *ov = oq + 4 * nb, *ow = ov + 3 * nb;
    for (int i = 0; i < nb; ++i) {
        if (w->props[i].type != FW_BODY_DYNAMIC) { mb[i] = 0.0f; continue; }
        for (int k = 0; k < 3; ++k) { op[3 * i + k] = xb[13 * i + k]; ov[3 * i + k] = xb[13 * i + 7 + k]; ow[3 * i + k] = xb[13 * i + 10 + k]; }
        for (int k = 0; k < 4; ++k) oq[4 * i + k] = xb[13 * i + 3 + k];
    }
    const cudaMemcpyKind out_kind = device_ptrs ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
    CK(cudaMemcpy(d_pos, op, sizeof(float) * 3 * nb, out_kind));
    CK(cudaMemcpy(d_quat, oq, sizeof(float) * 4 * nb, out_kind));
    CK(cudaMemcpy(d_linvel, ov, sizeof(float) * 3 * nb, out_kind));
    CK(cudaMemcpy(d_angvel, ow, sizeof(float) * 3 * nb, out_kind));
    CK(cudaMemcpy(d_mass, mb.data(), sizeof(float) * nb, out_kind));
    if (np > 0) CK(cudaMemcpy(d_mu, mub.data(), sizeof(float) * np, out_kind));
    return FW_OK;
}

fw_status fw_step_fwd_ckpt(fw_world *w, int n_substeps, int n_iters) {
    return fw_record_rollout(w, n_substeps, n_iters);
}

fw_status fw_step_bwd(fw_world *w, const float *g_pos, const float *g_quat, const float *g_linvel,
                      const float *g_angvel, float *d_pos, float *d_quat, float *d_linvel, float *d_angvel,
                      float *d_mass, float *d_mu, int device_ptrs) {
    return fw_adjoint_rollout(w, g_pos, g_quat, g_linvel, g_angvel, d_pos, d_quat, d_linvel, d_angvel, d_mass, d_mu,
                              device_ptrs);
}

fw_status fw_get_tape(fw_world *w, int info[4], int *c_off, int *c_rec, unsigned char *r_bits, unsigned char *b_bits) {
    if (!ready(w) || !info) return FW_ERR_ARG;
    if (!w->diff_valid) return fail(w, FW_ERR_STATE, "fw_get_tape: no recorded rollout");
    DiffState &d = w->diff;
    const int E = (int)w->envs.size();
    const size_t slots = (size_t)d.S * E;
    CK(cudaStreamSynchronize(w->stream));
    std::vector<int> tn(slots);
    CK(cudaMemcpy(tn.data(), d.tape_n, sizeof(int) * slots, cudaMemcpyDeviceToHost));
    long long total = 0;
    for (int v : tn) total += v;
    info[0] = d.S; info[1] = E; info[2] = d.K; info[3] = (int)total;
    if (!c_off || !c_rec || !r_bits || !b_bits) return FW_OK;
    const size_t rec_ints = diff_tape_record_bytes() / sizeof(int);
    std::vector<int> tc(slots * d.row_cap * rec_ints);
    std::vector<unsigned char> tr(slots * d.row_cap * (size_t)d.K), tb(slots);
    CK(cudaMemcpy(tc.data(), d.tape_c, sizeof(int) * tc.size(), cudaMemcpyDeviceToHost));
    if (!tr.empty()) CK(cudaMemcpy(tr.data(), d.tape_r, tr.size(), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(tb.data(), d.tape_b, slots, cudaMemcpyDeviceToHost));
    int c = 0;
    for (size_t sl = 0; sl < slots; ++sl) {
        c_off[sl] = c;
        for (int r = 0; r < tn[sl]; ++r, ++c) {
            for (size_t k = 0; k < 6; ++k) c_rec[6 * (size_t)c + k] = tc[(sl * d.row_cap + r) * rec_ints + k];
            for (int it = 0; it < d.K; ++it) r_bits[(size_t)d.K * c + it] = tr[(sl * d.row_cap + r) * d.K + it];
        }
        b_bits[sl] = tb[sl];
    }
    c_off[slots] = c;
    return FW_OK;
}

fw_status fw_get_detect_stats(fw_world *w, long long *n_candidates, long long *n_contacts) {
    if (!ready(w)) return FW_ERR_ARG;
    CK(cudaStreamSynchronize(w->stream));
    long long nc = 0, nk = 0;
    if (w->n_items > 0 && w->d_cand_count) {
        std::vector<int> c(w->n_items);
        CK(cudaMemcpy(c.data(), w->d_cand_count, sizeof(int) * w->n_items, cudaMemcpyDeviceToHost));
        for (int v : c) nc += v;
    }
    const int np = (int)w->pairs.size();
    if (np > 0 && w->d_counts) {
        std::vector<int> c(np);
        CK(cudaMemcpy(c.data(), w->d_counts, sizeof(int) * np, cudaMemcpyDeviceToHost));
        for (int v : c) nk += v;
    }
    for (size_t k = 0; k < w->piles.size(); ++k) {   // each pile: its items and pairs in use
        int2 c;
        CK(cudaMemcpy(&c, w->d_pcounts + k, sizeof c, cudaMemcpyDeviceToHost));
        std::vector<int> ci(c.y), cp(c.x);
        if (c.y > 0)
            CK(cudaMemcpy(ci.data(), w->d_pcand_count + k * w->pile_icap, sizeof(int) * c.y, cudaMemcpyDeviceToHost));
        if (c.x > 0)
            CK(cudaMemcpy(cp.data(), w->d_pccounts + k * w->pile_pcap, sizeof(int) * c.x, cudaMemcpyDeviceToHost));
        for (int v : ci) nc += v;
        for (int v : cp) nk += v;
    }
    if (n_candidates) *n_candidates = nc;
    if (n_contacts) *n_contacts = nk;
    return FW_OK;
}

fw_status fw_get_counts(fw_world *w, int *n_envs, int *n_bodies, int *n_pairs) {
    if (!w) return FW_ERR_ARG;
    if (n_envs) *n_envs = (int)w->envs.size();
    if (n_bodies) *n_bodies = (int)w->props.size();
    if (n_pairs) *n_pairs = (int)w->pairs.size();
    return FW_OK;
}

fw_status fw_get_env_info(fw_world *w, int env, int *first_body, int *n_bodies, int *first_pair, int *n_pairs) {
    if (!w) return FW_ERR_ARG;
    if (env < 0 || env >= (int)w->envs.size()) return fail(w, FW_ERR_ARG, "fw_get_env_info: env out of range");
    const EnvDev &E = w->envs[env];
    if (first_body) *first_body = E.first_body;
    if (n_bodies) *n_bodies = E.n_bodies;
    if (first_pair) *first_pair = E.pile >= 0 ? -1 : E.first_pair;
    if (n_pairs) *n_pairs = E.pile >= 0 ? -1 : E.n_pairs;
    return FW_OK;
}

fw_status fw_get_pile_pairs(fw_world *w, int env, int *pairs, int *colors, int cap, int *n_out) {
    if (!ready(w)) return FW_ERR_ARG;
    if (env < 0 || env >= (int)w->envs.size() || w->envs[env].pile < 0 || cap < 0 || (cap > 0 && !pairs) || !n_out)
        return fail(w, FW_ERR_ARG, "fw_get_pile_pairs: bad argument (env must be a pile env)");
    fw_status st = ensure_device(w);
    if (st != FW_OK) return st;
    const int k = w->envs[env].pile;
    int n = 0;
    if ((st = pile_pair_count(w, k, &n)) != FW_OK) return st;
    *n_out = n;
    const int m = std::min(n, cap);
    if (m > 0) {
        std::vector<PairDev> P(m);
        std::vector<unsigned char> c(m);
        CK(cudaMemcpy(P.data(), w->d_ppairs + (size_t)k * w->pile_pcap, sizeof(PairDev) * m, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(c.data(), w->pmem.color + (size_t)k * w->pile_pcap, m, cudaMemcpyDeviceToHost));
        for (int q = 0; q < m; ++q) {
            pairs[2 * q] = P[q].local_a;
            pairs[2 * q + 1] = P[q].local_b;
            if (colors) colors[q] = c[q] == 255 ? -1 : (int)c[q];
        }
    }
    st = check_status(w);
    if (st != FW_OK) return st;
    return n > cap ? fail(w, FW_ERR_OVERFLOW, "fw_get_pile_pairs: cap too small") : FW_OK;
}

int fw_launches_per_step(fw_world *w, int n_substeps) {
    if (!w || n_substeps < 1) return 0;
    // per substep: envs of listed pairs -- the pairs' maps (per-sample generation only),
    // query, reduction, solve; piles -- pair list, maps, query, reduction, the solve's prep
    // and its cooperative sweeps (kernels only: the barrier reset is a memset)
    const int regular = w->n_regular > 0 ? (w->cfg.contact_gen == 0 ? 4 : 3) : 0;
    return (regular + (w->piles.empty() ? 0 : 6)) * n_substeps;
}

const char *fw_last_error(const fw_world *w) {
    if (!w) return "null world";
    return w->err.c_str();
}

fw_status fw_measure_l2_read(int device, long long bytes, int iters, float *gbs) {
    if (!gbs || bytes < (1LL << 20) || bytes % 16 != 0 || iters < 1) return FW_ERR_ARG;
    return fw::measure_l2_read(device, bytes, iters, gbs) == cudaSuccess ? FW_OK : FW_ERR_CUDA;
}

}  // extern "C"
