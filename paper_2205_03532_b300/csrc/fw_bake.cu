// fw_bake.cu -- SDF generation from a triangle mesh (Sec. III-A: the SDF is sampled from
// the mesh once, at set-up).  Per grid node:
//   1. float32 search over all triangles (tiles staged in shared memory; a warp skips a
//      tile whose bounding box cannot beat any of its lanes' current candidates),
//      keeping the four nearest triangles;
//   2. float64 re-evaluation of those four (closest point and its feature: face, edge or
//      vertex), the nearest giving |phi|;
//   3. the sign from the angle-weighted pseudonormal of that feature (Baerentzen & Aanaes
//      2005), exact for closed manifold meshes; nodes where that test is within rounding
//      of zero are listed and get their sign from a float64 generalized winding number.
// Triangle distance: inside the prism over the face -> plane distance, else the nearest
// of the three edge segments.
#include "fw_device.cuh"

namespace fw {

namespace {

constexpr int kTile = 128;          // triangles per shared-memory tile
constexpr int kBakeThreads = 256;   // 8 x 8 x 4 node brick
constexpr int kTopK = 4;

struct TriF {
    float a[3], b[3], c[3];
};

// squared distance from p to segment a + t e, t in [0, 1]
__device__ __forceinline__ float seg_d2(V3 p, V3 a, V3 e) {
    const V3 d = p - a;
    const float ee = dot(e, e);
    const float t = ee > 0.0f ? fminf(fmaxf(dot(d, e) / ee, 0.0f), 1.0f) : 0.0f;
    const V3 r = d - t * e;
    return dot(r, r);
}

__device__ __forceinline__ float tri_d2_f32(V3 p, const TriF &T) {
    const V3 a = ld3(T.a), b = ld3(T.b), c = ld3(T.c);
    const V3 ab = b - a, bc = c - b, ca = a - c;
    const V3 n = cross(ab, c - a);
    const float s0 = dot(cross(ab, p - a), n);
    const float s1 = dot(cross(bc, p - b), n);
    const float s2 = dot(cross(ca, p - c), n);
    if (s0 >= 0.0f && s1 >= 0.0f && s2 >= 0.0f) {
        const float h = dot(p - a, n);
        return h * h / dot(n, n);
    }
    return fminf(seg_d2(p, a, ab), fminf(seg_d2(p, b, bc), seg_d2(p, c, ca)));
}

struct D3 {
    double x, y, z;
};
__device__ __forceinline__ D3 d3(double x, double y, double z) { return {x, y, z}; }
__device__ __forceinline__ D3 operator-(D3 a, D3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ D3 operator+(D3 a, D3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ D3 operator*(double s, D3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double ddot(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ D3 dcross(D3 a, D3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ D3 dload(const float *p) { return {(double)p[0], (double)p[1], (double)p[2]}; }

// float64 closest point on the triangle and its feature:
// 0 face, 1/2/3 vertex a/b/c, 4/5/6 edge ab/bc/ca
__device__ double tri_closest_f64(D3 p, const float *tri, D3 &q, int &feat) {
    const D3 a = dload(tri), b = dload(tri + 3), c = dload(tri + 6);
    const D3 ab = b - a, bc = c - b, ca = a - c;
    const D3 n = dcross(ab, c - a);
    const double s0 = ddot(dcross(ab, p - a), n);
    const double s1 = ddot(dcross(bc, p - b), n);
    const double s2 = ddot(dcross(ca, p - c), n);
    if (s0 >= 0.0 && s1 >= 0.0 && s2 >= 0.0) {
        const double h = ddot(p - a, n) / ddot(n, n);
        q = p - h * n;
        feat = 0;
        const D3 d = p - q;
        return ddot(d, d);
    }
    double best = 1e300;
    const D3 starts[3] = {a, b, c};
    const D3 edges[3] = {ab, bc, ca};
    for (int k = 0; k < 3; ++k) {
        const D3 d = p - starts[k];
        const double ee = ddot(edges[k], edges[k]);
        double t = ddot(d, edges[k]) / ee;
        int f = 4 + k;
        if (t <= 0.0) { t = 0.0; f = 1 + k; }
        else if (t >= 1.0) { t = 1.0; f = 1 + (k + 1) % 3; }
        const D3 qq = starts[k] + t * edges[k];
        const D3 r = p - qq;
        const double d2 = ddot(r, r);
        if (d2 < best) { best = d2; q = qq; feat = f; }
    }
    return best;
}

__device__ __forceinline__ void node_pos(const AssetDev &g, int i, int j, int k, double x[3]) {
    x[0] = (double)g.lo[0] + (double)i * (double)g.h;
    x[1] = (double)g.lo[1] + (double)j * (double)g.h;
    x[2] = (double)g.lo[2] + (double)k * (double)g.h;
}

__global__ void __launch_bounds__(kBakeThreads) bake_kernel(const float *tri, int nt, const float *tri_pn,
                                                            const float *tile_box, AssetDev g, float *out,
                                                            int *flags) {
    __shared__ TriF sT[kTile];
    const int bx = (g.dims[0] + 7) / 8, by = (g.dims[1] + 7) / 8;
    const int blk = blockIdx.x;
    const int bi = blk % bx, bj = (blk / bx) % by, bk = blk / (bx * by);
    const int t = threadIdx.x;
    const int i = bi * 8 + (t & 7), j = bj * 8 + ((t >> 3) & 7), k = bk * 4 + (t >> 6);
    const bool valid = i < g.dims[0] && j < g.dims[1] && k < g.dims[2];
    double xd[3];
    node_pos(g, i, j, k, xd);
    const V3 x = v3((float)xd[0], (float)xd[1], (float)xd[2]);
    float bd[kTopK];
    int bidx[kTopK];
    for (int q = 0; q < kTopK; ++q) { bd[q] = 3.0e38f; bidx[q] = -1; }
    const int n_tiles = (nt + kTile - 1) / kTile;
    for (int tile = 0; tile < n_tiles; ++tile) {
        // skip the tile when no lane can improve its k-th best
        const float *bb = tile_box + 6 * tile;
        const float dx = fmaxf(fmaxf(bb[0] - x.x, x.x - bb[3]), 0.0f);
        const float dy = fmaxf(fmaxf(bb[1] - x.y, x.y - bb[4]), 0.0f);
        const float dz = fmaxf(fmaxf(bb[2] - x.z, x.z - bb[5]), 0.0f);
        const float lb = (dx * dx + dy * dy + dz * dz) * 0.999f;
        const bool need = valid && lb <= bd[kTopK - 1];
        if (!__syncthreads_or(need)) continue;
        const int base = tile * kTile;
        const int cnt = min(kTile, nt - base);
        for (int q = t; q < cnt * 9; q += kBakeThreads) (&sT[0].a[0])[q] = tri[9 * base + q];
        __syncthreads();
        if (__any_sync(0xffffffffu, need)) {
            for (int q = 0; q < cnt; ++q) {
                const float d2 = tri_d2_f32(x, sT[q]);
                if (d2 < bd[kTopK - 1]) {
                    int s = kTopK - 1;
                    while (s > 0 && bd[s - 1] > d2) {
                        bd[s] = bd[s - 1];
                        bidx[s] = bidx[s - 1];
                        --s;
                    }
                    bd[s] = d2;
                    bidx[s] = base + q;
                }
            }
        }
        __syncthreads();
    }
    if (!valid) return;
    // float64 re-evaluation of the candidates
    const D3 p = d3(xd[0], xd[1], xd[2]);
    double best = 1e300;
    D3 qbest = p;
    int fbest = 0, tbest = -1;
    for (int q = 0; q < kTopK; ++q) {
        if (bidx[q] < 0) continue;
        D3 qq;
        int f;
        const double d2 = tri_closest_f64(p, tri + 9 * bidx[q], qq, f);
        if (d2 < best) { best = d2; qbest = qq; fbest = f; tbest = bidx[q]; }
    }
    const double dist = sqrt(best);
    const long long node = ((long long)k * g.dims[1] + j) * g.dims[0] + i;
    if (dist == 0.0 || tbest < 0) { out[node] = 0.0f; return; }
    // pseudonormal of the closest feature: slot 0 face, 1..3 edges ab/bc/ca, 4..6 vertices a/b/c
    const int slot = (fbest == 0) ? 0 : (fbest >= 4 ? fbest - 3 : fbest + 3);
    const float *N = tri_pn + 21 * tbest + 3 * slot;
    const D3 r = p - qbest;
    const double s = r.x * (double)N[0] + r.y * (double)N[1] + r.z * (double)N[2];
    if (fabs(s) <= 1e-6 * dist) {
        const int pos = atomicAdd(flags, 1);
        flags[1 + pos] = (int)node;   // sign resolved by the winding-number pass
        out[node] = (float)dist;
        return;
    }
    out[node] = (float)(s > 0.0 ? dist : -dist);
}

// Van Oosterom-Strackee solid angle of each triangle seen from the node, summed / 4 pi.
__global__ void winding_fix_kernel(const float *tri, int nt, AssetDev g, float *out, const int *idx, int n) {
    const int q = blockIdx.x;
    if (q >= n) return;
    const int node = idx[q];
    const int i = node % g.dims[0], j = (node / g.dims[0]) % g.dims[1], k = node / (g.dims[0] * g.dims[1]);
    double xd[3];
    node_pos(g, i, j, k, xd);
    const D3 p = d3(xd[0], xd[1], xd[2]);
    double acc = 0.0;
    for (int t = threadIdx.x; t < nt; t += blockDim.x) {
        const D3 A = dload(tri + 9 * t) - p, B = dload(tri + 9 * t + 3) - p, C = dload(tri + 9 * t + 6) - p;
        const double la = sqrt(ddot(A, A)), lb = sqrt(ddot(B, B)), lc = sqrt(ddot(C, C));
        const double num = ddot(A, dcross(B, C));
        const double den = la * lb * lc + ddot(A, B) * lc + ddot(B, C) * la + ddot(C, A) * lb;
        acc += 2.0 * atan2(num, den);
    }
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double wn = red[0] / (4.0 * 3.14159265358979323846);
        const float d = fabsf(out[node]);
        out[node] = (wn > 0.5) ? -d : d;
    }
}

// Corners of cell (i, j, k) of a node grid written as entry `dst` of a cell-corner copy
// (layout in AssetDev); float16 cells hold phi / h rounded to nearest.
__device__ __forceinline__ void write_cell(const float *grid, long long nx, long long nxy, long long i, long long j,
                                           long long k, float inv_h, float4 *c32, uint4 *c16, long long dst) {
    const float *b = grid + k * nxy + j * nx + i;
    const float v[8] = {b[0], b[1], b[nx], b[nx + 1], b[nxy], b[nxy + 1], b[nxy + nx], b[nxy + nx + 1]};
    if (c16) {
        unsigned u[4];
        for (int q = 0; q < 4; ++q) {
            const __half2 hh = __halves2half2(__float2half_rn(v[2 * q] * inv_h), __float2half_rn(v[2 * q + 1] * inv_h));
            u[q] = *reinterpret_cast<const unsigned *>(&hh);
        }
        c16[dst] = make_uint4(u[0], u[1], u[2], u[3]);
    } else {
        c32[2 * dst] = make_float4(v[0], v[1], v[2], v[3]);
        c32[2 * dst + 1] = make_float4(v[4], v[5], v[6], v[7]);
    }
}

// Dense cell-corner copy of a node grid: cell (i, j, k), i fastest.
__global__ void cells_kernel(const float *grid, int nx, int ny, int nz, float inv_h, float4 *c32, uint4 *c16) {
    const long long cnx = nx - 1, cny = ny - 1, n = cnx * cny * (long long)(nz - 1);
    const long long nxy = (long long)nx * ny;
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (; c < n; c += stride) {
        const long long i = c % cnx, j = (c / cnx) % cny, k = c / (cnx * cny);
        write_cell(grid, nx, nxy, i, j, k, inv_h, c32, c16, c);
    }
}

// Narrow band: one warp per brick reads the nodes of its cells (those of a partial brick
// at the grid's far faces stop at the last node) and flags it 1 if a node has |phi| <=
// band or the nodes change sign, else -1 (all above +band) or -2 (all below -band).
__global__ void brick_flags_kernel(const float *grid, int nx, int ny, int nz, float band, int bx, int by, int bz,
                                   int *flag) {
    const int lane = threadIdx.x & 31;
    const long long nb = (long long)bx * by * bz;
    const long long wpb = blockDim.x >> 5;
    const long long stride = (long long)gridDim.x * wpb;
    for (long long b = blockIdx.x * wpb + (threadIdx.x >> 5); b < nb; b += stride) {   // warp-uniform
        const int bi = (int)(b % bx), bj = (int)((b / bx) % by), bk = (int)(b / ((long long)bx * by));
        const int i0 = bi * kBrick, j0 = bj * kBrick, k0 = bk * kBrick;
        const int ni = min(i0 + kBrick, nx - 1) - i0 + 1, nj = min(j0 + kBrick, ny - 1) - j0 + 1;
        const int nk = min(k0 + kBrick, nz - 1) - k0 + 1;
        const int n = ni * nj * nk;
        bool near = false, pos = false, neg = false;
        for (int q = lane; q < n; q += 32) {
            const int i = i0 + q % ni, j = j0 + (q / ni) % nj, k = k0 + q / (ni * nj);
            const float v = grid[((long long)k * ny + j) * nx + i];
            near |= fabsf(v) <= band;
            if (v < 0.0f) neg = true; else pos = true;
        }
        near = __any_sync(0xffffffffu, near);
        pos = __any_sync(0xffffffffu, pos);
        neg = __any_sync(0xffffffffu, neg);
        if (lane == 0) flag[b] = (near || (pos && neg)) ? 1 : (neg ? -2 : -1);
    }
}

// Cell-corner copies of the stored bricks: cell (li, lj, lk) of slot s is entry
// s * kBrickCells + (lk * kBrick + lj) * kBrick + li; cells past the grid's last cell (a
// partial brick) are zero and never read.
__global__ void brick_cells_kernel(const float *grid, int nx, int ny, int nz, float inv_h, int bx, int by,
                                   const int *brick_of_slot, int n_stored, float4 *c32, uint4 *c16) {
    const long long n = (long long)n_stored * kBrickCells;
    const long long nxy = (long long)nx * ny;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
        const int b = brick_of_slot[t / kBrickCells];
        const int l = (int)(t % kBrickCells);
        const long long i = (long long)(b % bx) * kBrick + (l & (kBrick - 1));
        const long long j = (long long)((b / bx) % by) * kBrick + ((l >> kBrickLog) & (kBrick - 1));
        const long long k = (long long)(b / (bx * by)) * kBrick + (l >> (2 * kBrickLog));
        if (i >= nx - 1 || j >= ny - 1 || k >= nz - 1) {
            if (c16) c16[t] = make_uint4(0u, 0u, 0u, 0u);
            else { c32[2 * t] = make_float4(0.f, 0.f, 0.f, 0.f); c32[2 * t + 1] = make_float4(0.f, 0.f, 0.f, 0.f); }
            continue;
        }
        write_cell(grid, nx, nxy, i, j, k, inv_h, c32, c16, t);
    }
}

}  // namespace

cudaError_t launch_bake(const float *d_tri, int n_tri, const float *d_tri_pn, const float *d_tile_box,
                        const AssetDev &g, float *d_out, int *d_flags, cudaStream_t s) {
    const int bx = (g.dims[0] + 7) / 8, by = (g.dims[1] + 7) / 8, bz = (g.dims[2] + 3) / 4;
    const long long nblk = (long long)bx * by * bz;
    bake_kernel<<<(unsigned)nblk, kBakeThreads, 0, s>>>(d_tri, n_tri, d_tri_pn, d_tile_box, g, d_out, d_flags);
    return cudaGetLastError();
}

cudaError_t launch_bake_fix_sign(const float *d_tri, int n_tri, const AssetDev &g, float *d_out, const int *d_idx,
                                 int n_idx, cudaStream_t s) {
    if (n_idx <= 0) return cudaSuccess;
    winding_fix_kernel<<<n_idx, 256, 0, s>>>(d_tri, n_tri, g, d_out, d_idx, n_idx);
    return cudaGetLastError();
}

cudaError_t launch_cells(const float *grid, const int dims[3], float inv_h, float4 *cell32, uint4 *cell16,
                         cudaStream_t s) {
    cells_kernel<<<148 * 8, 256, 0, s>>>(grid, dims[0], dims[1], dims[2], inv_h, cell32, cell16);
    return cudaGetLastError();
}

cudaError_t launch_brick_flags(const float *grid, const int dims[3], float band, const int bdims[3], int *flags,
                               cudaStream_t s) {
    brick_flags_kernel<<<148 * 8, 256, 0, s>>>(grid, dims[0], dims[1], dims[2], band, bdims[0], bdims[1], bdims[2],
                                               flags);
    return cudaGetLastError();
}

cudaError_t launch_brick_cells(const float *grid, const int dims[3], float inv_h, const int bdims[3],
                               const int *brick_of_slot, int n_stored, float4 *cell32, uint4 *cell16, cudaStream_t s) {
    if (n_stored <= 0) return cudaSuccess;
    brick_cells_kernel<<<148 * 8, 256, 0, s>>>(grid, dims[0], dims[1], dims[2], inv_h, bdims[0], bdims[1],
                                               brick_of_slot, n_stored, cell32, cell16);
    return cudaGetLastError();
}

int bake_tile_size() { return kTile; }

}  // namespace fw
