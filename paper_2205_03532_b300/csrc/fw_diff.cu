// fw_diff.cu -- differentiable rollout on the device: a substep forward that records (or
// replays) each of its discrete decisions, and the reverse mode of that forward.
//
// Scope: an env takes part when exactly one of its bodies is dynamic and that body is the
// point-sampled body a of every pair of the env (its partners are static or kinematic:
// prescribed motion, no adjoint); envs with no dynamic body just move their kinematic
// bodies.  The forward of one env and substep:
//   external forces (gravity, applied force and torque, gyroscopic term) at the
//   substep's start; for each taped contact (sample of body a, pair, SDF cell of body b,
//   flags) the world point, the SDF value, gradient and Hessian of the taped cell's
//   trilinear polynomial, the normal and the contact rows (Sec. III-A, III-B);
//   K Gauss-Seidel sweeps of the normal row (lambda_n >= 0) and the jointly projected
//   friction rows, with the clamp and projection decisions taped per contact and sweep;
//   semi-implicit integration with an optional |omega| clamp (taped).
// Holding the decisions fixed makes the rollout a smooth function of the initial state,
// the dynamic body's mass (inertia scaled at fixed geometry) and the pairs' friction
// coefficients; the reverse kernel below is its exact reverse mode, run substep by
// substep from the last, each recomputing its forward from a checkpoint of the state at
// that substep's start.
//
// One warp per env, four envs per block.  Lane 0 runs the serial parts (sweeps,
// integration, their reverse); the lanes share the contacts for geometry and rows and
// their reverse, whose body-level sums are reduced in a fixed order (deterministic).
// For an env of at most kDiffSmemRows contacts the serial sweeps read the rows' solve
// coefficients, the impulses and the row adjoints from shared memory (the lanes stage
// them), and fetch the next update's recorded inputs and decision bits one step ahead;
// larger envs use the same code on the global copies.
#include "fw_device.cuh"

namespace fw {

namespace {

constexpr int kDiffWarps = 4;
constexpr int kDiffSmemRows = 128;  // contacts of an env whose sweeps run from shared memory


// (omega, 0) (x) q for q = (x, y, z, w)
__device__ __forceinline__ float4 omega_q(V3 w, float4 q) {
    return make_float4(q.w * w.x + w.y * q.z - w.z * q.y, q.w * w.y + w.z * q.x - w.x * q.z,
                       q.w * w.z + w.x * q.y - w.y * q.x, -(w.x * q.x + w.y * q.y + w.z * q.z));
}

__device__ __forceinline__ void mat_sym(const M3 &R, const float *S6, float *M9) {   // R S R^T, full 3x3
    float S[9] = {S6[0], S6[3], S6[4], S6[3], S6[1], S6[5], S6[4], S6[5], S6[2]};
    float T[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) T[3 * i + j] = R.m[3 * i] * S[j] + R.m[3 * i + 1] * S[3 + j] + R.m[3 * i + 2] * S[6 + j];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M9[3 * i + j] = T[3 * i] * R.m[3 * j] + T[3 * i + 1] * R.m[3 * j + 1] + T[3 * i + 2] * R.m[3 * j + 2];
}
__device__ __forceinline__ V3 mat9(const float *M, V3 v) {
    return v3(M[0] * v.x + M[1] * v.y + M[2] * v.z, M[3] * v.x + M[4] * v.y + M[5] * v.z, M[6] * v.x + M[7] * v.y + M[8] * v.z);
}
__device__ __forceinline__ V3 mat9t(const float *M, V3 v) {
    return v3(M[0] * v.x + M[3] * v.y + M[6] * v.z, M[1] * v.x + M[4] * v.y + M[7] * v.z, M[2] * v.x + M[5] * v.y + M[8] * v.z);
}

// cell fraction of x along one axis for a given cell c (same error-free parts as grid_coord)
__device__ __forceinline__ float grid_frac(float x, float lo, float inv_h, float inv_h_lo, int c) {
    const float s = x - lo;
    const float bb = s - x;
    const float e = (x - (s - bb)) + (-lo - bb);
    const float p = s * inv_h;
    const float pe = __fmaf_rn(s, inv_h, -p);
    const float corr = pe + __fmaf_rn(s, inv_h_lo, e * inv_h);
    return (p - (float)c) + corr;
}

// value, gradient and mixed second derivatives (xy, xz, yz) of cell c's trilinear
// polynomial at grid-frame x, world units; the diagonal of the Hessian is zero
__device__ void cell_eval(const AssetDev &g, const int c[3], V3 x, float &phi, V3 &grad, float H[3]) {
    const float fx = grid_frac(x.x, g.lo[0], g.inv_h, g.inv_h_lo, c[0]);
    const float fy = grid_frac(x.y, g.lo[1], g.inv_h, g.inv_h_lo, c[1]);
    const float fz = grid_frac(x.z, g.lo[2], g.inv_h, g.inv_h_lo, c[2]);
    int st;   // a taped cell made a candidate, so with narrow-band bricks its brick is stored
    const long long o = cell_offset<kStoreAny>(g, c[0], c[1], c[2], st);
    float v000, v100, v010, v110, v001, v101, v011, v111;
    if (g.cell16) {
        const uint4 q = g.cell16[o];
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&q.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&q.y));
        const float2 d = __half22float2(*reinterpret_cast<const __half2 *>(&q.z));
        const float2 e = __half22float2(*reinterpret_cast<const __half2 *>(&q.w));
        v000 = a.x; v100 = a.y; v010 = b.x; v110 = b.y; v001 = d.x; v101 = d.y; v011 = e.x; v111 = e.y;
    } else {
        const float4 a = g.cell32[2 * o], b = g.cell32[2 * o + 1];
        v000 = a.x; v100 = a.y; v010 = a.z; v110 = a.w; v001 = b.x; v101 = b.y; v011 = b.z; v111 = b.w;
    }
    const float a00 = lerp_(v000, v100, fx), a10 = lerp_(v010, v110, fx);
    const float a01 = lerp_(v001, v101, fx), a11 = lerp_(v011, v111, fx);
    const float val = lerp_(lerp_(a00, a10, fy), lerp_(a01, a11, fy), fz);
    const float gx = lerp_(lerp_(v100 - v000, v110 - v010, fy), lerp_(v101 - v001, v111 - v011, fy), fz);
    const float gy = lerp_(lerp_(v010 - v000, v110 - v100, fx), lerp_(v011 - v001, v111 - v101, fx), fz);
    const float gz = lerp_(lerp_(v001 - v000, v101 - v100, fx), lerp_(v011 - v010, v111 - v110, fx), fy);
    const float hxy = lerp_((v110 - v010) - (v100 - v000), (v111 - v011) - (v101 - v001), fz);
    const float hxz = lerp_((v101 - v001) - (v100 - v000), (v111 - v011) - (v110 - v010), fy);
    const float hyz = lerp_((v011 - v001) - (v010 - v000), (v111 - v101) - (v110 - v100), fx);
    // node values are phi (float32 copy) or phi / h (float16 copy)
    const float sv = g.cell16 ? g.h : 1.0f, sg = g.cell16 ? 1.0f : g.inv_h;
    const float sh = g.cell16 ? g.inv_h : g.inv_h * g.inv_h;
    phi = val * sv;
    grad = v3(gx * sg, gy * sg, gz * sg);
    H[0] = hxy * sh; H[1] = hxz * sh; H[2] = hyz * sh;
}

struct TapeC {
    int sample, pair, ci, cj, ck, flags;   // flags: bit 0 t1 from n x e_x, bit 1 phi > 0
};

struct DRow {   // one contact row of the dynamic body, world frame
    float s[3];
    int cell[3], flags, pair, live;
    float xbl[3], phi, g[3], gn, H[3], nb[3];
    float xa[3], xbw[3], n[3];
    float ra[3], rb[3], uo[3], tr[3], tn;
    float d[3][3], a[3][3], b[3][3], k[3];
    float bias, e[3], mu;
};

struct __align__(16) DRowBar {   // 144 bytes: nine float4
    float d[3][3], a[3][3], b[3][3], k[3], bias, e[3], mu;
};

// the fields of a DRow that one row update reads (160 bytes: ten float4)
struct __align__(16) SRow {
    float d[3][3], a[3][3], b[3][3], k[3], bias, e[3], mu;
    int live, pad_[2];
};

// shared memory of one env (one warp)
struct EnvSmem {
    SRow row[kDiffSmemRows];
    float lam[3 * kDiffSmemRows];      // impulses (forward), their adjoints (reverse)
    DRowBar bar[kDiffSmemRows];        // row adjoints (reverse)
};

struct St {
    float *pos, *quat, *lin, *ang;
};

struct DiffParams {
    SimParams p;
    int S, K, si, row_cap, record;
    float hs;
    const int *dyn;           // per env: dynamic body (global id) or -1
    TapeC *tape_c;            // (S * n_envs) x row_cap
    int *tape_n;              // S * n_envs
    unsigned char *tape_r;    // (S * n_envs * row_cap) x K
    unsigned char *tape_b;    // S * n_envs
    St ck;                    // S blocks of n_bodies states (state at each substep's start)
    St scratch;               // n_bodies (recomputed states that are not kept)
    DRow *rows;               // n_envs x row_cap
    DRowBar *rbar;            // n_envs x row_cap
    float *upd;               // n_envs x row_cap x K x 9
    float *lam;               // n_envs x row_cap x 3 (impulses; adjoints of impulses in reverse)
    float *xb;                // n_bodies x 13 adjoint state (pos 3, quat 4, lin 3, ang 3)
    float *mass_b;            // n_bodies
    float *mu_row;            // n_envs x row_cap
    float *mu_b;              // n_pairs
};

struct DBody {   // body-level forward intermediates of one env substep
    float4 q0, qt, q1;
    M3 R;
    float Iw[9], Ii[9];
    V3 com, v0, w0, v1, w1, Lw, tq, vf, wf, wc;
    int clamped;
};

__device__ __forceinline__ float4 ldq(const float *q, int b) { return make_float4(q[4 * b], q[4 * b + 1], q[4 * b + 2], q[4 * b + 3]); }
__device__ __forceinline__ void stq(float *q, int b, float4 v) { q[4 * b] = v.x; q[4 * b + 1] = v.y; q[4 * b + 2] = v.z; q[4 * b + 3] = v.w; }

// geometry and rows of one taped contact
__device__ void build_drow(const DiffParams &dp, const St &in, const DBody &F, const BodyProps &PA, int ia, DRow &D) {
    const SimParams &p = dp.p;
    const PairDev P = p.pairs[D.pair];
    const int ib = P.b;
    const AssetDev gb = p.assets[P.asset_b];
    const M3 RB = quat_to_mat(ldq(in.quat, ib));
    const V3 pB = ld3(in.pos + 3 * ib);
    const V3 xa = mul(F.R, ld3(D.s)) + ld3(in.pos + 3 * ia);
    const V3 xbl = mul_t(RB, xa - pB);
    float phi, H[3];
    V3 g;
    cell_eval(gb, D.cell, xbl, phi, g, H);
    const float gn = sqrtf(dot(g, g));
    const V3 nb = (1.0f / gn) * g;
    const V3 n = mul(RB, nb);
    const V3 xbw = xa - phi * n;
    const V3 ra = xa - F.com;
    const BodyProps PB = p.props[ib];
    const V3 comB = mul(RB, ld3(PB.com_b)) + pB;
    const V3 rb = xbw - comB;
    const V3 uo = ld3(in.lin + 3 * ib) + cross(ld3(in.ang + 3 * ib), rb);
    const V3 tr = (D.flags & 1) ? v3(0.f, n.z, -n.y) : v3(-n.z, 0.f, n.x);
    const float tn = sqrtf(dot(tr, tr));
    const V3 t1 = (1.0f / tn) * tr;
    const V3 t2 = cross(n, t1);
    st3(D.xbl, xbl); D.phi = phi; st3(D.g, g); D.gn = gn;
    D.H[0] = H[0]; D.H[1] = H[1]; D.H[2] = H[2];
    st3(D.nb, nb); st3(D.xa, xa); st3(D.xbw, xbw); st3(D.n, n);
    st3(D.ra, ra); st3(D.rb, rb); st3(D.uo, uo); st3(D.tr, tr); D.tn = tn;
    const V3 dd[3] = {n, t1, t2};
    D.live = 1;
    for (int j = 0; j < 3; ++j) {
        const V3 a = cross(ra, dd[j]);
        const V3 b = mat9(F.Ii, a);
        st3(D.d[j], dd[j]); st3(D.a[j], a); st3(D.b[j], b);
        const float den = PA.invm + dot(a, b);
        D.k[j] = den > 0.0f ? 1.0f / den : 0.0f;
        D.e[j] = -dot(dd[j], uo);
    }
    if (D.k[0] == 0.0f) D.live = 0;
    D.bias = (D.flags & 2) ? phi / dp.hs : p.baumgarte * phi / dp.hs;
    D.mu = P.mu;
}

// one row update with the given decisions (replay: taken from `taped`; record: computed
// and written to *bits)
template <class R>
__device__ __forceinline__ void drow_fwd(const R &D, float invm, V3 &v, V3 &w, float *lam, unsigned char taped,
                                         unsigned char *bits, bool replay) {
    const float jv = dot(ld3(D.d[0]), v) + dot(ld3(D.a[0]), w) + D.bias + D.e[0];
    const float u = lam[0] - D.k[0] * jv;
    const bool act = replay ? ((taped & 1) != 0) : (u > 0.0f);
    const float ln = act ? u : 0.0f;
    const float dl = ln - lam[0];
    const V3 vm = v + (invm * dl) * ld3(D.d[0]);
    const V3 wm = w + dl * ld3(D.b[0]);
    const float j1 = dot(ld3(D.d[1]), vm) + dot(ld3(D.a[1]), wm) + D.e[1];
    const float j2 = dot(ld3(D.d[2]), vm) + dot(ld3(D.a[2]), wm) + D.e[2];
    const float t1 = lam[1] - D.k[1] * j1, t2 = lam[2] - D.k[2] * j2;
    const float lim = D.mu * ln, tn = sqrtf(t1 * t1 + t2 * t2);
    const bool proj = replay ? ((taped & 2) != 0) : (tn > lim);
    const float s = proj ? lim / tn : 1.0f;
    const float l1 = s * t1, l2 = s * t2;
    const float e1 = l1 - lam[1], e2 = l2 - lam[2];
    v = vm + invm * (e1 * ld3(D.d[1]) + e2 * ld3(D.d[2]));
    w = wm + e1 * ld3(D.b[1]) + e2 * ld3(D.b[2]);
    lam[0] = ln; lam[1] = l1; lam[2] = l2;
    if (!replay) *bits = (unsigned char)((act ? 1 : 0) | (proj ? 2 : 0));
}

// K sweeps over nr rows, as lane 0 runs them: the taped decision bit of the next row is
// loaded a step ahead (replay); upd, when not NULL, receives each update's inputs.
template <class R>
__device__ void sweeps_fwd(const R *rows, int nr, int K, float invm, V3 &v, V3 &w, float *L, unsigned char *bits,
                           bool replay, float *upd) {
    if (nr == 0) return;
    unsigned char next = replay ? bits[0] : 0;
    for (int it = 0; it < K; ++it)
        for (int r = 0; r < nr; ++r) {
            const unsigned char taped = next;
            if (replay) {
                const int rn = (r + 1 < nr) ? r + 1 : 0, itn = (r + 1 < nr) ? it : it + 1;
                if (itn < K) next = bits[(size_t)rn * K + itn];
            }
            if (upd) {
                float *u = upd + ((size_t)r * K + it) * 9;
                u[0] = v.x; u[1] = v.y; u[2] = v.z; u[3] = w.x; u[4] = w.y; u[5] = w.z;
                u[6] = L[3 * r]; u[7] = L[3 * r + 1]; u[8] = L[3 * r + 2];
            }
            if (!rows[r].live) continue;
            const R D = rows[r];
            drow_fwd(D, invm, v, w, L + 3 * r, taped, bits + (size_t)r * K + it, replay);
        }
}

// Forward of env e in substep dp.si from state `in`; writes the new state to `out` (which
// may be `in`: every input is read first).  keep: store each update's inputs in dp.upd.
// sm: the warp's shared memory (NULL: rows, impulses from global memory).
__device__ void env_forward(const DiffParams &dp, int e, int lane, const St &in, const St &out, bool replay,
                            bool keep, DBody &F, EnvSmem *sm) {
    const SimParams &p = dp.p;
    const EnvDev E = p.envs[e];
    const int ia = dp.dyn[e];
    const int slot = dp.si * p.n_envs + e;
    const float hs = dp.hs;
    F.clamped = 0;
    if (ia >= 0) {
        const BodyProps PA = p.props[ia];
        F.q0 = ldq(in.quat, ia);
        F.R = quat_to_mat(F.q0);
        mat_sym(F.R, PA.Ib, F.Iw);
        mat_sym(F.R, PA.Ib_inv, F.Ii);
        F.com = mul(F.R, ld3(PA.com_b)) + ld3(in.pos + 3 * ia);
        F.v0 = ld3(in.lin + 3 * ia);
        F.w0 = ld3(in.ang + 3 * ia);
        const V3 gv = v3(p.gravity[0], p.gravity[1], p.gravity[2]);
        F.v1 = F.v0 + hs * (gv + (1.0f / PA.mass) * ld3(PA.force));
        F.Lw = mat9(F.Iw, F.w0);
        F.tq = ld3(PA.torque) - cross(F.w0, F.Lw);
        F.w1 = F.w0 + hs * mat9(F.Ii, F.tq);
        // contacts of this substep: from detection (record) or from the tape (replay)
        TapeC *tc = dp.tape_c + (size_t)slot * dp.row_cap;
        int nr;
        if (!replay) {
            int acc = 0;
            for (int k = 0; k < E.n_pairs; ++k) {
                const int pi = E.first_pair + k;
                const int cnt = min(p.counts[pi], p.cap_pair);
                const PairDev P = p.pairs[pi];
                const AssetDev gb = p.assets[P.asset_b];
                const M3 RB = quat_to_mat(ldq(in.quat, P.b));
                const V3 pB = ld3(in.pos + 3 * P.b);
                for (int i = lane; i < cnt; i += 32) {
                    const int r = acc + i;
                    if (r >= dp.row_cap) continue;
                    const int sm = p.contacts[(long long)pi * p.cap_pair + i].sample_patch & 0xFFFFFF;
                    const float4 s4 = p.assets[P.asset_a].samples[sm];
                    const V3 xa = mul(F.R, v3(s4.x, s4.y, s4.z)) + ld3(in.pos + 3 * ia);
                    const V3 xbl = mul_t(RB, xa - pB);
                    int c[3];
                    float f;
                    grid_coord(xbl.x, gb.lo[0], gb.inv_h, gb.inv_h_lo, gb.dims[0], c[0], f);
                    grid_coord(xbl.y, gb.lo[1], gb.inv_h, gb.inv_h_lo, gb.dims[1], c[1], f);
                    grid_coord(xbl.z, gb.lo[2], gb.inv_h, gb.inv_h_lo, gb.dims[2], c[2], f);
                    float phi, H[3];
                    V3 g;
                    cell_eval(gb, c, xbl, phi, g, H);
                    const V3 n = mul(RB, (1.0f / sqrtf(dot(g, g))) * g);
                    TapeC t;
                    t.sample = sm; t.pair = pi; t.ci = c[0]; t.cj = c[1]; t.ck = c[2];
                    t.flags = (fabsf(n.x) < 0.57735f ? 1 : 0) | (phi > 0.0f ? 2 : 0);
                    tc[r] = t;
                }
                acc += cnt;
            }
            nr = min(acc, dp.row_cap);
            if (lane == 0) dp.tape_n[slot] = nr;
            __syncwarp();
        } else {
            nr = dp.tape_n[slot];
        }
        DRow *rows = dp.rows + (size_t)e * dp.row_cap;
        for (int r = lane; r < nr; r += 32) {
            const TapeC t = tc[r];
            DRow D;
            const float4 s4 = p.assets[p.pairs[t.pair].asset_a].samples[t.sample];
            D.s[0] = s4.x; D.s[1] = s4.y; D.s[2] = s4.z;
            D.cell[0] = t.ci; D.cell[1] = t.cj; D.cell[2] = t.ck;
            D.flags = t.flags; D.pair = t.pair;
            build_drow(dp, in, F, PA, ia, D);
            rows[r] = D;
        }
        __threadfence_block();
        __syncwarp();
        const bool staged = sm && nr <= kDiffSmemRows;
        if (staged) {   // the rows' solve coefficients and zero impulses into shared memory
            for (int r = lane; r < nr; r += 32) {
                const DRow &D = rows[r];
                SRow &Sr = sm->row[r];
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) { Sr.d[i][j] = D.d[i][j]; Sr.a[i][j] = D.a[i][j]; Sr.b[i][j] = D.b[i][j]; }
                for (int i = 0; i < 3; ++i) { Sr.k[i] = D.k[i]; Sr.e[i] = D.e[i]; }
                Sr.bias = D.bias; Sr.mu = D.mu; Sr.live = D.live;
                sm->lam[3 * r] = 0.f; sm->lam[3 * r + 1] = 0.f; sm->lam[3 * r + 2] = 0.f;
            }
            __syncwarp();
        }
        // sweeps and integration on lane 0
        if (lane == 0) {
            V3 v = F.v1, w = F.w1;
            float *L = staged ? sm->lam : dp.lam + (size_t)e * dp.row_cap * 3;   // impulses, no warm start
            if (!staged)
                for (int r = 0; r < nr; ++r) { L[3 * r] = 0.f; L[3 * r + 1] = 0.f; L[3 * r + 2] = 0.f; }
            unsigned char *bits = dp.tape_r + (size_t)slot * dp.row_cap * dp.K;
            float *upd = keep ? dp.upd + (size_t)e * dp.row_cap * dp.K * 9 : nullptr;
            if (staged)
                sweeps_fwd(sm->row, nr, dp.K, PA.invm, v, w, L, bits, replay, upd);
            else
                sweeps_fwd(rows, nr, dp.K, PA.invm, v, w, L, bits, replay, upd);
            F.vf = v;
            F.wf = w;
            const float wn = sqrtf(dot(w, w));
            if (!replay) dp.tape_b[slot] = (p.max_angvel > 0.0f && wn > p.max_angvel) ? 1 : 0;
            F.clamped = dp.tape_b[slot] & 1;
            F.wc = F.clamped ? (p.max_angvel / wn) * w : w;
            const V3 cp = F.com + hs * F.vf;
            const float4 dq = omega_q(F.wc, F.q0);
            const float hh = 0.5f * hs;
            F.qt = make_float4(F.q0.x + hh * dq.x, F.q0.y + hh * dq.y, F.q0.z + hh * dq.z, F.q0.w + hh * dq.w);
            const float inv = 1.0f / sqrtf(F.qt.x * F.qt.x + F.qt.y * F.qt.y + F.qt.z * F.qt.z + F.qt.w * F.qt.w);
            F.q1 = make_float4(F.qt.x * inv, F.qt.y * inv, F.qt.z * inv, F.qt.w * inv);
            const M3 R1 = quat_to_mat(F.q1);
            const V3 pn = cp - mul(R1, ld3(PA.com_b));
            st3(out.pos + 3 * ia, pn);
            stq(out.quat, ia, F.q1);
            st3(out.lin + 3 * ia, F.vf);
            st3(out.ang + 3 * ia, F.wc);
        }
    }
    // kinematic bodies follow their prescribed velocity; static ones stay
    for (int lb = lane; lb < E.n_bodies; lb += 32) {
        const int bi = E.first_body + lb;
        if (bi == ia) continue;
        const BodyProps P = p.props[bi];
        const V3 pos = ld3(in.pos + 3 * bi), v = ld3(in.lin + 3 * bi), w = ld3(in.ang + 3 * bi);
        const float4 q = ldq(in.quat, bi);
        if (P.type != FW_BODY_KINEMATIC) {
            st3(out.pos + 3 * bi, pos); stq(out.quat, bi, q); st3(out.lin + 3 * bi, v); st3(out.ang + 3 * bi, w);
            continue;
        }
        const M3 R = quat_to_mat(q);
        const V3 cp = mul(R, ld3(P.com_b)) + pos + hs * v;
        const float4 dq = omega_q(w, q);
        const float hh = 0.5f * hs;
        float4 qt = make_float4(q.x + hh * dq.x, q.y + hh * dq.y, q.z + hh * dq.z, q.w + hh * dq.w);
        const float inv = 1.0f / sqrtf(qt.x * qt.x + qt.y * qt.y + qt.z * qt.z + qt.w * qt.w);
        qt = make_float4(qt.x * inv, qt.y * inv, qt.z * inv, qt.w * inv);
        const V3 pn = cp - mul(quat_to_mat(qt), ld3(P.com_b));
        st3(out.pos + 3 * bi, pn); stq(out.quat, bi, qt); st3(out.lin + 3 * bi, v); st3(out.ang + 3 * bi, w);
    }
    __syncwarp();
}


// ---------------------------------------------------------------------------- reverse
// adjoint of R = quat_to_mat(q): the derivative of each entry's polynomial in (x, y, z, w)
__device__ float4 quat_mat_vjp(float4 q, const float Rb[9]) {
    const float x = q.x, y = q.y, z = q.z, w = q.w;
    float4 g;
    g.x = 2.f * (y * Rb[1] + z * Rb[2] + y * Rb[3] - w * Rb[5] + z * Rb[6] + w * Rb[7]) - 4.f * x * (Rb[4] + Rb[8]);
    g.y = 2.f * (x * Rb[1] + w * Rb[2] + x * Rb[3] + z * Rb[5] - w * Rb[6] + z * Rb[7]) - 4.f * y * (Rb[0] + Rb[8]);
    g.z = 2.f * (-w * Rb[1] + x * Rb[2] + w * Rb[3] + y * Rb[5] + x * Rb[6] + y * Rb[7]) - 4.f * z * (Rb[0] + Rb[4]);
    g.w = 2.f * (-z * Rb[1] + y * Rb[2] + z * Rb[3] - x * Rb[5] - y * Rb[6] + x * Rb[7]);
    return g;
}

__device__ __forceinline__ void outer_add(float *M, V3 a, V3 b, float s = 1.0f) {   // M += s a b^T
    M[0] += s * a.x * b.x; M[1] += s * a.x * b.y; M[2] += s * a.x * b.z;
    M[3] += s * a.y * b.x; M[4] += s * a.y * b.y; M[5] += s * a.y * b.z;
    M[6] += s * a.z * b.x; M[7] += s * a.z * b.y; M[8] += s * a.z * b.z;
}

__device__ __forceinline__ void add3(float *a, V3 b) { a[0] += b.x; a[1] += b.y; a[2] += b.z; }

// reverse of drow_fwd: u = (v, w, lambda) before the update; vb, wb, lb: adjoints of the
// outputs in, of the inputs out; the row's data adjoints accumulate in X
template <class R>
__device__ __forceinline__ void drow_rev(const R &D, float invm, const float *u, unsigned char bits, V3 &vb, V3 &wb,
                                         float *lb, DRowBar &X, float &invm_b) {
    const V3 v = v3(u[0], u[1], u[2]), w = v3(u[3], u[4], u[5]);
    const float lam0 = u[6], lam1 = u[7], lam2 = u[8];
    const V3 d0 = ld3(D.d[0]), d1 = ld3(D.d[1]), d2 = ld3(D.d[2]);
    const V3 a0 = ld3(D.a[0]), a1 = ld3(D.a[1]), a2 = ld3(D.a[2]);
    const V3 b0 = ld3(D.b[0]), b1 = ld3(D.b[1]), b2 = ld3(D.b[2]);
    const float jv = dot(d0, v) + dot(a0, w) + D.bias + D.e[0];
    const float uu = lam0 - D.k[0] * jv;
    const bool act = bits & 1, proj = (bits & 2) != 0;
    const float ln = act ? uu : 0.0f, dl = ln - lam0;
    const V3 vm = v + (invm * dl) * d0, wm = w + dl * b0;
    const float j1 = dot(d1, vm) + dot(a1, wm) + D.e[1];
    const float j2 = dot(d2, vm) + dot(a2, wm) + D.e[2];
    const float t1 = lam1 - D.k[1] * j1, t2 = lam2 - D.k[2] * j2;
    const float lim = D.mu * ln, tn = sqrtf(t1 * t1 + t2 * t2);
    const float s = proj ? lim / tn : 1.0f;
    const float e1 = s * t1 - lam1, e2 = s * t2 - lam2;
    // v' = vm + invm (e1 d1 + e2 d2), w' = wm + e1 b1 + e2 b2
    V3 vmb = vb, wmb = wb;
    const float e1b = invm * dot(d1, vb) + dot(b1, wb);
    const float e2b = invm * dot(d2, vb) + dot(b2, wb);
    add3(X.d[1], (invm * e1) * vb); add3(X.d[2], (invm * e2) * vb);
    add3(X.b[1], e1 * wb); add3(X.b[2], e2 * wb);
    invm_b += e1 * dot(vb, d1) + e2 * dot(vb, d2);
    // e_k = s t_k - lambda_k
    const float l1b = lb[1] + e1b, l2b = lb[2] + e2b;
    float lam1b = -e1b, lam2b = -e2b;
    float t1b = s * l1b, t2b = s * l2b, lnb = lb[0];
    if (proj) {   // s = lim / |t|
        const float sb = t1 * l1b + t2 * l2b;
        const float limb = sb / tn, tnb = -sb * lim / (tn * tn);
        t1b += tnb * t1 / tn;
        t2b += tnb * t2 / tn;
        X.mu += ln * limb;
        lnb += D.mu * limb;
    }
    // t_k = lambda_k - k_k j_k
    lam1b += t1b;
    lam2b += t2b;
    X.k[1] -= j1 * t1b;
    X.k[2] -= j2 * t2b;
    const float j1b = -D.k[1] * t1b, j2b = -D.k[2] * t2b;
    // j_k = d_k . vm + a_k . wm + e_k
    vmb = vmb + j1b * d1 + j2b * d2;
    wmb = wmb + j1b * a1 + j2b * a2;
    add3(X.d[1], j1b * vm); add3(X.d[2], j2b * vm);
    add3(X.a[1], j1b * wm); add3(X.a[2], j2b * wm);
    X.e[1] += j1b;
    X.e[2] += j2b;
    // vm = v + invm dl d0, wm = w + dl b0
    const float dlb = invm * dot(d0, vmb) + dot(b0, wmb);
    add3(X.d[0], (invm * dl) * vmb);
    add3(X.b[0], dl * wmb);
    invm_b += dl * dot(d0, vmb);
    // dl = ln - lambda_0;  ln = u (taped active) or 0;  u = lambda_0 - k_0 jv
    lnb += dlb;
    float lam0b = -dlb;
    const float ub = act ? lnb : 0.0f;
    lam0b += ub;
    X.k[0] -= jv * ub;
    const float jvb = -D.k[0] * ub;
    vb = vmb + jvb * d0;
    wb = wmb + jvb * a0;
    add3(X.d[0], jvb * v);
    add3(X.a[0], jvb * w);
    X.bias += jvb;
    X.e[0] += jvb;
    lb[0] = lam0b; lb[1] = lam1b; lb[2] = lam2b;
}

// Body-level sums gathered from the contacts in the reverse of one substep.
struct BodyBar {
    float comb[3], Iib[9], invm_b, pb[3], Rb[9];
};

// reverse of the contact geometry and rows of one contact (lanes in parallel)
__device__ void drow_prep_rev(const DiffParams &dp, const DBody &F, const St &in, const DRow &D, const DRowBar &X,
                              BodyBar &B) {
    const SimParams &p = dp.p;
    const int ib = p.pairs[D.pair].b;
    float ab[3][3], bb[3][3], db[3][3];
    for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) { ab[j][i] = X.a[j][i]; bb[j][i] = X.b[j][i]; db[j][i] = X.d[j][i]; }
    V3 rab = v3(0, 0, 0), uob = v3(0, 0, 0);
    for (int j = 0; j < 3; ++j) {
        const float denb = -D.k[j] * D.k[j] * X.k[j];   // k = 1 / den, den = invm + a . b
        B.invm_b += denb;
        const V3 a = ld3(D.a[j]), b = ld3(D.b[j]), d = ld3(D.d[j]);
        V3 abv = ld3(ab[j]) + denb * b;
        const V3 bbv = ld3(bb[j]) + denb * a;
        abv = abv + mat9t(F.Ii, bbv);                    // b = Ii a
        outer_add(B.Iib, bbv, a);
        uob = uob - X.e[j] * d;                          // e = -d . uo
        V3 dbv = ld3(db[j]) - X.e[j] * ld3(D.uo);
        rab = rab + cross(d, abv);                       // a = ra x d
        dbv = dbv + cross(abv, ld3(D.ra));
        db[j][0] = dbv.x; db[j][1] = dbv.y; db[j][2] = dbv.z;
    }
    float phib = X.bias * ((D.flags & 2) ? 1.0f / dp.hs : p.baumgarte / dp.hs);
    const V3 wB = ld3(in.ang + 3 * ib);
    const V3 rbb = cross(uob, wB);                       // uo = vB + wB x rb
    const V3 xbwb = rbb;                                 // rb = xbw - comB
    V3 xab = rab;                                        // ra = xa - com
    B.comb[0] -= rab.x; B.comb[1] -= rab.y; B.comb[2] -= rab.z;
    // d0 = n, d1 = tr / |tr|, d2 = n x d1
    const V3 n = ld3(D.n), d1 = ld3(D.d[1]);
    V3 nbv = ld3(db[0]) + cross(d1, ld3(db[2]));
    const V3 d1b = ld3(db[1]) + cross(ld3(db[2]), n);
    const V3 trb = (1.0f / D.tn) * (d1b - dot(d1, d1b) * d1);
    if (D.flags & 1) { nbv.z += trb.y; nbv.y -= trb.z; }
    else { nbv.z -= trb.x; nbv.x += trb.z; }
    // xbw = xa - phi n
    xab = xab + xbwb;
    nbv = nbv - D.phi * xbwb;
    phib -= dot(n, xbwb);
    // n = RB nb, nb = g / |g|
    const M3 RB = quat_to_mat(ldq(in.quat, ib));
    const V3 nbb = mul_t(RB, nbv);
    const V3 nb = ld3(D.nb);
    const V3 gb = (1.0f / D.gn) * (nbb - dot(nb, nbb) * nb);
    // (phi, g) of the taped cell at xbl: xbl_b = g phi_b + H g_b
    const V3 xblb = phib * ld3(D.g) + v3(D.H[0] * gb.y + D.H[1] * gb.z, D.H[0] * gb.x + D.H[2] * gb.z,
                                         D.H[1] * gb.x + D.H[2] * gb.y);
    // xbl = RB^T (xa - pB), xa = R s + p
    const V3 xwb = mul(RB, xblb) + xab;
    add3(B.pb, xwb);
    outer_add(B.Rb, xwb, ld3(D.s));
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Reverse of one env substep; the forward (with keep) has just run from `in`.
// The sweeps of one env in reverse, as lane 0 runs them: last update first, the next
// update's recorded inputs and decision bits loaded a step ahead.
template <class R>
__device__ void sweeps_rev(const R *rows, DRowBar *X, int nr, int K, float invm, const float *upd,
                           const unsigned char *bits, V3 &vb, V3 &wb, float *lb, float &invm_b) {
    if (nr == 0 || K == 0) return;
    int it = K - 1, r = nr - 1;
    float un[9];
    unsigned char bn = bits[(size_t)r * K + it];
    for (int k = 0; k < 9; ++k) un[k] = upd[((size_t)r * K + it) * 9 + k];
    for (;;) {
        float u[9];
        for (int k = 0; k < 9; ++k) u[k] = un[k];
        const unsigned char b = bn;
        const int rc = r;
        if (--r < 0) { r = nr - 1; --it; }
        if (it >= 0) {
            bn = bits[(size_t)r * K + it];
            for (int k = 0; k < 9; ++k) un[k] = upd[((size_t)r * K + it) * 9 + k];
        }
        if (rows[rc].live) {   // the row and its adjoints in registers for the update
            const R D = rows[rc];
            DRowBar Xr = X[rc];
            drow_rev(D, invm, u, b, vb, wb, lb + 3 * rc, Xr, invm_b);
            X[rc] = Xr;
        }
        if (it < 0) break;
    }
}

__device__ void env_reverse(const DiffParams &dp, int e, int lane, const St &in, const DBody &F, EnvSmem *sm) {
    const SimParams &p = dp.p;
    const int ia = dp.dyn[e];
    const BodyProps PA = p.props[ia];
    const int slot = dp.si * p.n_envs + e;
    const int nr = dp.tape_n[slot];
    DRow *rows = dp.rows + (size_t)e * dp.row_cap;
    // the forward just ran (env_forward with keep) and staged the rows when this holds
    const bool staged = sm && nr <= kDiffSmemRows;
    DRowBar *rbar = staged ? sm->bar : dp.rbar + (size_t)e * dp.row_cap;
    float *lb = staged ? sm->lam : dp.lam + (size_t)e * dp.row_cap * 3;
    float *xb = dp.xb + 13 * ia;
    const float hs = dp.hs;
    for (int r = lane; r < nr; r += 32) {
        DRowBar z;
        memset(&z, 0, sizeof z);
        rbar[r] = z;
        lb[3 * r] = 0.f; lb[3 * r + 1] = 0.f; lb[3 * r + 2] = 0.f;
    }
    __threadfence_block();
    __syncwarp();
    // ---- serial part on lane 0: integration, sweeps
    float invm_b0 = 0.0f;
    V3 v1b = v3(0, 0, 0), w1b = v3(0, 0, 0), comb0 = v3(0, 0, 0);
    float4 qb0 = make_float4(0, 0, 0, 0);
    if (lane == 0) {
        const V3 pb = ld3(xb);
        float4 qb1 = make_float4(xb[3], xb[4], xb[5], xb[6]);
        V3 vb = ld3(xb + 7), wcb = ld3(xb + 10);
        // p' = c' - R(q') com_b
        float R1b[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        outer_add(R1b, pb, ld3(PA.com_b), -1.0f);
        const float4 g1 = quat_mat_vjp(F.q1, R1b);
        qb1.x += g1.x; qb1.y += g1.y; qb1.z += g1.z; qb1.w += g1.w;
        // q' = qt / |qt|
        const float qn = sqrtf(F.qt.x * F.qt.x + F.qt.y * F.qt.y + F.qt.z * F.qt.z + F.qt.w * F.qt.w);
        const float dq = F.q1.x * qb1.x + F.q1.y * qb1.y + F.q1.z * qb1.z + F.q1.w * qb1.w;
        const float4 tb = make_float4((qb1.x - F.q1.x * dq) / qn, (qb1.y - F.q1.y * dq) / qn,
                                      (qb1.z - F.q1.z * dq) / qn, (qb1.w - F.q1.w * dq) / qn);
        // qt = q + hs/2 (wc, 0) (x) q
        const float hh = 0.5f * hs;
        const float4 q = F.q0;
        const V3 wc = F.wc;
        qb0 = make_float4(tb.x + hh * (wc.z * tb.y - wc.y * tb.z - wc.x * tb.w),
                          tb.y + hh * (-wc.z * tb.x + wc.x * tb.z - wc.y * tb.w),
                          tb.z + hh * (wc.y * tb.x - wc.x * tb.y - wc.z * tb.w),
                          tb.w + hh * (wc.x * tb.x + wc.y * tb.y + wc.z * tb.z));
        wcb = wcb + hh * v3(q.w * tb.x - q.z * tb.y + q.y * tb.z - q.x * tb.w,
                            q.z * tb.x + q.w * tb.y - q.x * tb.z - q.y * tb.w,
                            -q.y * tb.x + q.x * tb.y + q.w * tb.z - q.z * tb.w);
        // c' = com + hs vf
        comb0 = pb;
        vb = vb + hs * pb;
        // |omega| clamp
        V3 wb = wcb;
        if (F.clamped) {
            const float wn = sqrtf(dot(F.wf, F.wf));
            const V3 uh = (1.0f / wn) * F.wf;
            wb = (p.max_angvel / wn) * (wcb - dot(uh, wcb) * uh);
        }
        // sweeps, last update first
        const unsigned char *bits = dp.tape_r + (size_t)slot * dp.row_cap * dp.K;
        const float *upd = dp.upd + (size_t)e * dp.row_cap * dp.K * 9;
        if (staged)
            sweeps_rev(sm->row, rbar, nr, dp.K, PA.invm, upd, bits, vb, wb, lb, invm_b0);
        else
            sweeps_rev(rows, rbar, nr, dp.K, PA.invm, upd, bits, vb, wb, lb, invm_b0);
        v1b = vb;
        w1b = wb;
    }
    __threadfence_block();
    __syncwarp();
    // ---- contacts in parallel, then a fixed-order warp reduction
    BodyBar B;
    memset(&B, 0, sizeof B);
    for (int r = lane; r < nr; r += 32) {
        const DRow D = rows[r];
        const DRowBar X = rbar[r];
        dp.mu_row[(size_t)e * dp.row_cap + r] = D.live ? X.mu : 0.0f;
        if (D.live) drow_prep_rev(dp, F, in, D, X, B);
    }
    float *bf = reinterpret_cast<float *>(&B);
    for (int k = 0; k < (int)(sizeof(BodyBar) / sizeof(float)); ++k) bf[k] = warp_sum(bf[k]);
    __threadfence_block();
    __syncwarp();
    if (lane != 0) return;
    // ---- external forces: v1 = v + hs (g + F/m), w1 = w + hs Ii (tau - w x Iw w)
    const float m = PA.mass;
    float mass_b = -hs * dot(ld3(PA.force), v1b) / (m * m);
    const V3 tqb = hs * mat9t(F.Ii, w1b);
    outer_add(B.Iib, w1b, F.tq, hs);
    const V3 gyb = -1.0f * tqb;                           // tq = tau - w x Lw
    V3 w0b = w1b + cross(F.Lw, gyb);                      // gy = w x Lw
    const V3 Lwb = cross(gyb, F.w0);
    w0b = w0b + mat9t(F.Iw, Lwb);                         // Lw = Iw w
    float Iwb[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    outer_add(Iwb, Lwb, F.w0);
    // com = R com_b + p
    const V3 comb = comb0 + ld3(B.comb);
    const V3 pb0 = ld3(B.pb) + comb;
    outer_add(B.Rb, comb, ld3(PA.com_b));
    // Iw = R Ib R^T, Ii = R Ib^-1 R^T:  Rb += (M_b + M_b^T) R S;  S_b = R^T M_b R
    const float Ib9[9] = {PA.Ib[0], PA.Ib[3], PA.Ib[4], PA.Ib[3], PA.Ib[1], PA.Ib[5], PA.Ib[4], PA.Ib[5], PA.Ib[2]};
    const float Ii9[9] = {PA.Ib_inv[0], PA.Ib_inv[3], PA.Ib_inv[4], PA.Ib_inv[3], PA.Ib_inv[1], PA.Ib_inv[5],
                          PA.Ib_inv[4], PA.Ib_inv[5], PA.Ib_inv[2]};
    float sIb = 0.f, sIi = 0.f;
    for (int which = 0; which < 2; ++which) {
        const float *Mb = which ? B.Iib : Iwb;
        const float *S = which ? Ii9 : Ib9;
        float Ms[9], T[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) Ms[3 * i + j] = Mb[3 * i + j] + Mb[3 * j + i];
        for (int i = 0; i < 3; ++i)   // T = Ms R
            for (int j = 0; j < 3; ++j)
                T[3 * i + j] = Ms[3 * i] * F.R.m[j] + Ms[3 * i + 1] * F.R.m[3 + j] + Ms[3 * i + 2] * F.R.m[6 + j];
        for (int i = 0; i < 3; ++i)   // Rb += T S
            for (int j = 0; j < 3; ++j) B.Rb[3 * i + j] += T[3 * i] * S[j] + T[3 * i + 1] * S[3 + j] + T[3 * i + 2] * S[6 + j];
        // <R^T Mb R, S> = <Mb, R S R^T>
        const float *RSR = which ? F.Ii : F.Iw;
        float acc = 0.f;
        for (int k = 0; k < 9; ++k) acc += Mb[k] * RSR[k];
        if (which) sIi = acc; else sIb = acc;
    }
    const float invm_b = invm_b0 + B.invm_b;
    mass_b += sIb / m - sIi / m - invm_b / (m * m);
    const float4 gq = quat_mat_vjp(F.q0, B.Rb);
    xb[0] = pb0.x; xb[1] = pb0.y; xb[2] = pb0.z;
    xb[3] = qb0.x + gq.x; xb[4] = qb0.y + gq.y; xb[5] = qb0.z + gq.z; xb[6] = qb0.w + gq.w;
    xb[7] = v1b.x; xb[8] = v1b.y; xb[9] = v1b.z;
    xb[10] = w0b.x; xb[11] = w0b.y; xb[12] = w0b.z;
    dp.mass_b[ia] += mass_b;
    for (int r = 0; r < nr; ++r) dp.mu_b[rows[r].pair] += dp.mu_row[(size_t)e * dp.row_cap + r];
}

__device__ __forceinline__ St ck_at(const DiffParams &dp, int s, int nb) {
    const size_t S = (size_t)dp.S;
    St c;
    c.pos = dp.ck.pos + (size_t)s * nb * 3;
    c.quat = dp.ck.pos + S * nb * 3 + (size_t)s * nb * 4;
    c.lin = dp.ck.pos + S * nb * 7 + (size_t)s * nb * 3;
    c.ang = dp.ck.pos + S * nb * 10 + (size_t)s * nb * 3;
    return c;
}

__global__ void __launch_bounds__(32 * kDiffWarps) diff_forward_kernel(DiffParams dp, int n_bodies, int replay) {
    const int e = blockIdx.x * kDiffWarps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (e >= dp.p.n_envs) return;
    const SimParams &p = dp.p;
    const EnvDev E = p.envs[e];
    const St world = {p.pos, p.quat, p.linvel, p.angvel};
    const St ck = ck_at(dp, dp.si, n_bodies);
    for (int lb = lane; lb < E.n_bodies; lb += 32) {   // checkpoint of the substep's start
        const int bi = E.first_body + lb;
        for (int k = 0; k < 3; ++k) {
            ck.pos[3 * bi + k] = p.pos[3 * bi + k];
            ck.lin[3 * bi + k] = p.linvel[3 * bi + k];
            ck.ang[3 * bi + k] = p.angvel[3 * bi + k];
        }
        for (int k = 0; k < 4; ++k) ck.quat[4 * bi + k] = p.quat[4 * bi + k];
    }
    __syncwarp();
    extern __shared__ EnvSmem diff_smem[];
    DBody F;
    env_forward(dp, e, lane, world, world, replay != 0, false, F, diff_smem + (threadIdx.x >> 5));
}

__global__ void __launch_bounds__(32 * kDiffWarps) diff_reverse_kernel(DiffParams dp, int n_bodies) {
    const int e = blockIdx.x * kDiffWarps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (e >= dp.p.n_envs) return;
    const St ck = ck_at(dp, dp.si, n_bodies);
    extern __shared__ EnvSmem diff_smem[];
    EnvSmem *sm = diff_smem + (threadIdx.x >> 5);
    DBody F;
    env_forward(dp, e, lane, ck, dp.scratch, true, true, F, sm);
    if (dp.dyn[e] >= 0) env_reverse(dp, e, lane, ck, F, sm);
}

constexpr size_t kDiffSmemBytes = sizeof(EnvSmem) * kDiffWarps;

// raise the kernels' dynamic shared-memory limit once per device (the block needs more
// than the default 48 KB)
cudaError_t prepare_diff_kernels() {
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(diff_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDiffSmemBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(diff_reverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDiffSmemBytes);
    if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
    return e;
}

DiffParams make_params(const SimParams &p, const DiffState &d, int si, int n_bodies) {
    DiffParams dp;
    dp.p = p;
    dp.S = d.S; dp.K = d.K; dp.si = si; dp.row_cap = d.row_cap; dp.record = 0;
    dp.hs = d.hs;
    dp.dyn = d.dyn;
    dp.tape_c = static_cast<TapeC *>(d.tape_c);
    dp.tape_n = d.tape_n;
    dp.tape_r = d.tape_r;
    dp.tape_b = d.tape_b;
    dp.ck = St{d.ck, nullptr, nullptr, nullptr};
    dp.scratch = St{d.scratch, d.scratch + 3 * (size_t)n_bodies, d.scratch + 7 * (size_t)n_bodies,
                    d.scratch + 10 * (size_t)n_bodies};
    dp.rows = static_cast<DRow *>(d.rows);
    dp.rbar = static_cast<DRowBar *>(d.rbar);
    dp.upd = d.upd; dp.lam = d.lam; dp.xb = d.xb; dp.mass_b = d.mass_b; dp.mu_row = d.mu_row; dp.mu_b = d.mu_b;
    return dp;
}

}  // namespace

size_t diff_tape_record_bytes() { return sizeof(TapeC); }
size_t diff_row_bytes() { return sizeof(DRow); }
size_t diff_row_bar_bytes() { return sizeof(DRowBar); }

cudaError_t launch_diff_forward(const SimParams &p, const DiffState &d, int si, int n_bodies, bool replay,
                                cudaStream_t s) {
    if (p.n_envs == 0) return cudaSuccess;
    const DiffParams dp = make_params(p, d, si, n_bodies);
    cudaError_t e = prepare_diff_kernels();
    if (e != cudaSuccess) return e;
    diff_forward_kernel<<<(p.n_envs + kDiffWarps - 1) / kDiffWarps, 32 * kDiffWarps, kDiffSmemBytes, s>>>(
        dp, n_bodies, replay ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_diff_reverse(const SimParams &p, const DiffState &d, int si, int n_bodies, cudaStream_t s) {
    if (p.n_envs == 0) return cudaSuccess;
    const DiffParams dp = make_params(p, d, si, n_bodies);
    cudaError_t e = prepare_diff_kernels();
    if (e != cudaSuccess) return e;
    diff_reverse_kernel<<<(p.n_envs + kDiffWarps - 1) / kDiffWarps, 32 * kDiffWarps, kDiffSmemBytes, s>>>(dp, n_bodies);
    return cudaGetLastError();
}

}  // namespace fw
