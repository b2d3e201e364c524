// fw_device.cuh -- device helpers: small vector algebra, quaternions, the SDF lookup.
#pragma once

#include "fw_internal.h"

namespace fw {

struct V3 {
    float x, y, z;
};
__device__ __forceinline__ V3 v3(float x, float y, float z) { return {x, y, z}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 operator*(float s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ float dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ V3 ld3(const float *p) { return {p[0], p[1], p[2]}; }
__device__ __forceinline__ void st3(float *p, V3 a) { p[0] = a.x; p[1] = a.y; p[2] = a.z; }

// Row-major 3x3 rotation of the unit quaternion q = (x, y, z, w).
struct M3 {
    float m[9];
};
__device__ __forceinline__ M3 quat_to_mat(float4 q) {
    float x = q.x, y = q.y, z = q.z, w = q.w;
    M3 R;
    R.m[0] = 1.f - 2.f * (y * y + z * z); R.m[1] = 2.f * (x * y - z * w);       R.m[2] = 2.f * (x * z + y * w);
    R.m[3] = 2.f * (x * y + z * w);       R.m[4] = 1.f - 2.f * (x * x + z * z); R.m[5] = 2.f * (y * z - x * w);
    R.m[6] = 2.f * (x * z - y * w);       R.m[7] = 2.f * (y * z + x * w);       R.m[8] = 1.f - 2.f * (x * x + y * y);
    return R;
}
__device__ __forceinline__ V3 mul(const M3 &R, V3 v) {
    return {R.m[0] * v.x + R.m[1] * v.y + R.m[2] * v.z, R.m[3] * v.x + R.m[4] * v.y + R.m[5] * v.z,
            R.m[6] * v.x + R.m[7] * v.y + R.m[8] * v.z};
}
__device__ __forceinline__ V3 mul_t(const M3 &R, V3 v) {   // R^T v
    return {R.m[0] * v.x + R.m[3] * v.y + R.m[6] * v.z, R.m[1] * v.x + R.m[4] * v.y + R.m[7] * v.z,
            R.m[2] * v.x + R.m[5] * v.y + R.m[8] * v.z};
}
// symmetric matrix stored xx yy zz xy xz yz
__device__ __forceinline__ V3 sym_mul(const float *S, V3 v) {
    return {S[0] * v.x + S[3] * v.y + S[4] * v.z, S[3] * v.x + S[1] * v.y + S[5] * v.z,
            S[4] * v.x + S[5] * v.y + S[2] * v.z};
}
// R S R^T for symmetric S (result symmetric, stored the same way)
__device__ __forceinline__ void rot_sym(const M3 &R, const float *S, float *out) {
    float T[9];  // R S
    for (int i = 0; i < 3; ++i) {
        V3 r = v3(R.m[3 * i], R.m[3 * i + 1], R.m[3 * i + 2]);
        V3 c = sym_mul(S, r);   // (S r)^T = r^T S (S symmetric)
        T[3 * i] = c.x; T[3 * i + 1] = c.y; T[3 * i + 2] = c.z;
    }
    auto e = [&](int i, int j) {
        return T[3 * i] * R.m[3 * j] + T[3 * i + 1] * R.m[3 * j + 1] + T[3 * i + 2] * R.m[3 * j + 2];
    };
    out[0] = e(0, 0); out[1] = e(1, 1); out[2] = e(2, 2);
    out[3] = e(0, 1); out[4] = e(0, 2); out[5] = e(1, 2);
}

// Tangent basis of a unit normal: t1 = normalize(n x e_x) when |n_x| < 0.57735, else
// normalize(n x e_y); t2 = n x t1.
__device__ __forceinline__ void tangent_basis(V3 n, V3 &t1, V3 &t2) {
    V3 t = (fabsf(n.x) < 0.57735f) ? v3(0.f, n.z, -n.y) : v3(-n.z, 0.f, n.x);
    float inv = 1.0f / sqrtf(dot(t, t));
    t1 = inv * t;
    t2 = cross(n, t1);
}

// ----------------------------------------------------------------------------------------
// SDF lookup (Sec. III-A): trilinear value and the analytic gradient of the trilinear
// interpolant.  The grid coordinate u = (x - lo) / h is formed as an unevaluated sum
// p + corr (TwoSum for x - lo, FMA residual for the product, and the float32 residual of
// 1/h), so the cell fraction is exact to float32 rounding of f itself instead of carrying
// the ~N * 2^-24 voxel error of a plain float32 (x - lo) * inv_h.
// ----------------------------------------------------------------------------------------
// Returns whether x lies in [lo, lo + (dim-1) h]; c, f are always usable (clamped to a
// cell of the grid), so callers can load the corners before knowing the answer.
__device__ __forceinline__ bool grid_coord(float x, float lo, float inv_h, float inv_h_lo, int dim,
                                           int &c, float &f) {
    const float s = x - lo;
    const float bb = s - x;
    const float e = (x - (s - bb)) + (-lo - bb);     // s + e == x - lo exactly
    const float p = s * inv_h;
    const float pe = __fmaf_rn(s, inv_h, -p);        // s * inv_h - p exactly
    const float corr = pe + __fmaf_rn(s, inv_h_lo, e * inv_h);
    bool ok = (p > -2.0f && p < (float)dim + 1.0f);  // also rejects NaN
    const float pc = ok ? p : 0.0f;
    float fl = floorf(pc);
    float fr = (pc - fl) + (ok ? corr : 0.0f);
    if (fr < 0.0f) { fl -= 1.0f; fr += 1.0f; }
    else if (fr >= 1.0f) { fl += 1.0f; fr -= 1.0f; }
    int ci = (int)fl;
    ok = ok && ci >= 0 && ci <= dim - 1 && !(ci == dim - 1 && fr > 0.0f);
    if (ci >= dim - 1) { ci = dim - 2; fr = 1.0f; }
    if (ci < 0) { ci = 0; fr = 0.0f; }
    c = ci;
    f = fr;
    return ok;
}

__device__ __forceinline__ float lerp_(float a, float b, float t) { return __fmaf_rn(t, b - a, a); }

// Storage of the cell-corner copies a lookup is compiled for: dense, narrow-band bricks,
// or either, decided per asset at run time.
enum : int { kStoreDense = 0, kStoreBricks = 1, kStoreAny = 2 };

// Entry of cell (ci, cj, ck) in the asset's cell-corner copy: dense (x fastest), or with
// narrow-band bricks the cell's place in its brick's slot.  st: the brick's table entry
// (0 when dense); st < 0 means the brick is not stored, and the entry returned is then a
// valid dummy (0) so that the load can still be issued unconditionally.
template <int kStore = kStoreAny>
__device__ __forceinline__ long long cell_offset(const AssetDev &g, int ci, int cj, int ck, int &st) {
    if (kStore == kStoreDense || (kStore == kStoreAny && !g.brick)) {
        st = 0;
        const long long cnx = g.dims[0] - 1, cnxy = cnx * (long long)(g.dims[1] - 1);
        return (long long)ck * cnxy + (long long)cj * cnx + ci;
    }
    st = __ldg(g.brick + ((ck >> kBrickLog) * g.bdims[1] + (cj >> kBrickLog)) * g.bdims[0] + (ci >> kBrickLog));
    const int l = ((ck & (kBrick - 1)) << (2 * kBrickLog)) | ((cj & (kBrick - 1)) << kBrickLog) | (ci & (kBrick - 1));
    return st >= 0 ? (long long)st * kBrickCells + l : 0;
}

// The 8 corner values of cell (ci, cj, ck) (order 000 100 010 110 001 101 011 111, x
// fastest; phi / h in FP16 storage) and the brick's table entry st (< 0: left out).
struct CellCorners {
    float v[8];
    int st;
};
template <bool kHalf, int kStore = kStoreAny>
__device__ __forceinline__ CellCorners sdf_cell_corners(const AssetDev &g, int ci, int cj, int ck) {
    CellCorners c;
    const long long o = cell_offset<kStore>(g, ci, cj, ck, c.st);
    if (kHalf) {
        const uint4 q = __ldg(g.cell16 + o);
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&q.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&q.y));
        const float2 d = __half22float2(*reinterpret_cast<const __half2 *>(&q.z));
        const float2 e = __half22float2(*reinterpret_cast<const __half2 *>(&q.w));
        c.v[0] = a.x; c.v[1] = a.y; c.v[2] = b.x; c.v[3] = b.y;
        c.v[4] = d.x; c.v[5] = d.y; c.v[6] = e.x; c.v[7] = e.y;
    } else {
        const float4 a = __ldg(g.cell32 + 2 * o), b = __ldg(g.cell32 + 2 * o + 1);
        c.v[0] = a.x; c.v[1] = a.y; c.v[2] = a.z; c.v[3] = a.w;
        c.v[4] = b.x; c.v[5] = b.y; c.v[6] = b.z; c.v[7] = b.w;
    }
    return c;
}
// The trilinear value of a cell's corners (the same lerps as sdf_cell_eval), in metres;
// +-band for a brick left out.
template <bool kHalf>
__device__ __forceinline__ float cell_value(const AssetDev &g, const CellCorners &c, float fx, float fy, float fz) {
    const float a00 = lerp_(c.v[0], c.v[1], fx), a10 = lerp_(c.v[2], c.v[3], fx);
    const float a01 = lerp_(c.v[4], c.v[5], fx), a11 = lerp_(c.v[6], c.v[7], fx);
    const float b0 = lerp_(a00, a10, fy), b1 = lerp_(a01, a11, fy);
    const float val = lerp_(b0, b1, fz);
    const float phi = kHalf ? val * g.h : val;
    return c.st < 0 ? (c.st == -1 ? g.band : -g.band) : phi;
}
// The gradient of the trilinear interpolant (the same blends as sdf_cell_eval); zero for a
// brick left out.
template <bool kHalf>
__device__ __forceinline__ V3 cell_gradient(const AssetDev &g, const CellCorners &c, float fx, float fy, float fz) {
    const float *v = c.v;
    const float gx = lerp_(lerp_(v[1] - v[0], v[3] - v[2], fy), lerp_(v[5] - v[4], v[7] - v[6], fy), fz);
    const float gy = lerp_(lerp_(v[2] - v[0], v[3] - v[1], fx), lerp_(v[6] - v[4], v[7] - v[5], fx), fz);
    const float gz = lerp_(lerp_(v[4] - v[0], v[5] - v[1], fx), lerp_(v[6] - v[2], v[7] - v[3], fx), fy);
    const V3 gr = kHalf ? v3(gx, gy, gz) : g.inv_h * v3(gx, gy, gz);
    return c.st < 0 ? v3(0.0f, 0.0f, 0.0f) : gr;
}

// Trilinear value and gradient in cell (ci, cj, ck) at fractions (fx, fy, fz) from the
// cell-corner copy (the cell must be a valid cell of the grid: its one or two 16-byte loads
// are in bounds).  A cell of a brick left out of the narrow band answers phi = +band (or
// -band inside) with a zero gradient.
template <bool kHalf, int kStore = kStoreAny>
__device__ __forceinline__ void sdf_cell_eval(const AssetDev &g, int ci, int cj, int ck, float fx, float fy, float fz,
                                              float &phi, V3 &grad) {
    int st;
    const long long o = cell_offset<kStore>(g, ci, cj, ck, st);
    float v000, v100, v010, v110, v001, v101, v011, v111;
    if (kHalf) {
        const uint4 c = __ldg(g.cell16 + o);
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&c.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&c.y));
        const float2 d = __half22float2(*reinterpret_cast<const __half2 *>(&c.z));
        const float2 e = __half22float2(*reinterpret_cast<const __half2 *>(&c.w));
        v000 = a.x; v100 = a.y; v010 = b.x; v110 = b.y;
        v001 = d.x; v101 = d.y; v011 = e.x; v111 = e.y;
    } else {
        const float4 a = __ldg(g.cell32 + 2 * o), b = __ldg(g.cell32 + 2 * o + 1);
        v000 = a.x; v100 = a.y; v010 = a.z; v110 = a.w;
        v001 = b.x; v101 = b.y; v011 = b.z; v111 = b.w;
    }
    // value: lerp along x, then y, then z
    const float a00 = lerp_(v000, v100, fx), a10 = lerp_(v010, v110, fx);
    const float a01 = lerp_(v001, v101, fx), a11 = lerp_(v011, v111, fx);
    const float b0 = lerp_(a00, a10, fy), b1 = lerp_(a01, a11, fy);
    const float val = lerp_(b0, b1, fz);
    // gradient: bilinear blend of the node differences along each axis
    const float gx = lerp_(lerp_(v100 - v000, v110 - v010, fy), lerp_(v101 - v001, v111 - v011, fy), fz);
    const float gy = lerp_(lerp_(v010 - v000, v110 - v100, fx), lerp_(v011 - v001, v111 - v101, fx), fz);
    const float gz = lerp_(lerp_(v001 - v000, v101 - v100, fx), lerp_(v011 - v010, v111 - v110, fx), fy);
    if (kHalf) {   // cells hold phi / h
        phi = val * g.h;
        grad = v3(gx, gy, gz);
    } else {
        phi = val;
        grad = g.inv_h * v3(gx, gy, gz);
    }
    if (st < 0) {
        phi = st == -1 ? g.band : -g.band;
        grad = v3(0.0f, 0.0f, 0.0f);
    }
}

// Trilinear value and gradient of the asset's SDF at x (grid frame); the corner loads are
// always in bounds and issued before the in-grid test is used, so several lookups can
// overlap their memory latency.  Returns whether x lies in the grid box.
template <bool kHalf, int kStore = kStoreAny>
__device__ __forceinline__ bool sdf_lookup(const AssetDev &g, V3 x, float &phi, V3 &grad) {
    int ci, cj, ck;
    float fx, fy, fz;
    const bool okx = grid_coord(x.x, g.lo[0], g.inv_h, g.inv_h_lo, g.dims[0], ci, fx);
    const bool oky = grid_coord(x.y, g.lo[1], g.inv_h, g.inv_h_lo, g.dims[1], cj, fy);
    const bool okz = grid_coord(x.z, g.lo[2], g.inv_h, g.inv_h_lo, g.dims[2], ck, fz);
    sdf_cell_eval<kHalf, kStore>(g, ci, cj, ck, fx, fy, fz, phi, grad);
    return okx && oky && okz;
}

// Cell index and fraction along one axis from a grid coordinate given as an integer part
// (exact) plus a float32 remainder u (|u| a few hundred at most): the cell holding the point
// clamped to the grid, and whether the point lies in [0, dim - 1].  NaN gives false.
__device__ __forceinline__ bool cell_of(float u, int base, int dim, int &c, float &f) {
    const float fl = floorf(u);
    float fr = u - fl;                                   // exact
    const bool finite = fl == fl && fabsf(fl) < 1.0e6f;
    int ci = finite ? (int)fl + base : -1;
    bool ok = finite && ci >= 0 && ci <= dim - 1 && !(ci == dim - 1 && fr > 0.0f);
    if (ci >= dim - 1) { ci = dim - 2; fr = 1.0f; }
    if (ci < 0) { ci = 0; fr = 0.0f; }
    c = ci;
    f = fr;
    return ok;
}

template <int kStore = kStoreAny>
__device__ __forceinline__ bool sdf_lookup_any(const AssetDev &g, V3 x, float &phi, V3 &grad) {
    return g.cell16 ? sdf_lookup<true, kStore>(g, x, phi, grad) : sdf_lookup<false, kStore>(g, x, phi, grad);
}

// Order-preserving map of a float to uint32 (larger float -> larger integer).
__device__ __forceinline__ unsigned ord_f32(float f) {
    f = f + 0.0f;   // -0 -> +0
    unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

}  // namespace fw
