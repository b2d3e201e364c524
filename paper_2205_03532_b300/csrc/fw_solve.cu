// fw_solve.cu -- contact solution of one substep (Sec. III-B): external forces,
// constraint preparation, Gauss-Seidel sweeps with Coulomb friction, integration.
// A group of lanes per environment (a whole warp, or 16, 8 or 4 lanes when several envs
// share a warp): its lanes prepare rows and integrate bodies in parallel; the sweep itself is
// the serial Gauss-Seidel chain, run with identical values by every lane of the group.
//
// Two sweep forms compute the same update.  Fast form (an env with at most one movable
// body, i.e. every other body static or kinematic): each contact is written from the
// movable body's side (directions negated when it is the pair's SDF body, the partner's
// prescribed velocity folded into a constant), 9 float4 per contact; the body's velocity
// stays in registers, the rows stream from global memory through a cp.async ring in
// shared memory and the accumulated impulses live in shared memory.  General form
// (several movable bodies): full two-body rows, velocities in shared memory, one lane.
//
// Update rule (velocity-level projected Gauss-Seidel; the paper cites the solver without
// restating it): per contact, the normal row
//     lambda_n <- max(0, lambda_n - k_n (n . v_rel + b)),
// then both friction rows from the updated velocities, lambda_t <- lambda_t - k_t (t . v_rel),
// projected jointly on the disk |lambda_t| <= mu lambda_n; every change is applied to
// both bodies at once.  b = phi/hs for phi > 0 (speculative contact), baumgarte*phi/hs
// otherwise.  Integration: semi-implicit Euler of the centre of mass and
// q <- normalize(q + hs/2 (omega, 0) q).
#include "fw_device.cuh"

namespace fw {

namespace {

constexpr int kMaxBodies = 8;
constexpr int kRing = 16;     // rows in flight in the fast sweep's shared-memory ring
constexpr int kRowF4 = 9;     // float4 per fast row
constexpr int kRowBlock = 2;  // fast rows solved between two warp barriers



__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

struct BodySm {
    float v[kMaxBodies][3], w[kMaxBodies][3];
    float invm[kMaxBodies];
    float Iinv[kMaxBodies][6];
    float com[kMaxBodies][3];
};

struct EnvSm {
    BodySm B;
    float q_new[kMaxBodies][4];
    int row_base[kMaxPairsPerEnv + 1];
};

// Dynamic shared memory of one env slot, in float4: impulse words, then the ring; padded to
// 1 mod 8 so that the envs of a warp, which read the same ring slot at the same time, start
// in different shared-memory banks.  The slot's bodies and row offsets (EnvSm) are in a
// static array of the kernel.
__host__ __device__ inline int env_stride_f4(int lam_cap) { return ((lam_cap + kRing * kRowF4 + 7) & ~7) + 1; }

__device__ __forceinline__ V3 smv(const float (*a)[3], int i) { return v3(a[i][0], a[i][1], a[i][2]); }
__device__ __forceinline__ void smv_set(float (*a)[3], int i, V3 x) { a[i][0] = x.x; a[i][1] = x.y; a[i][2] = x.z; }

// effective mass 1 / (m_a^-1 + m_b^-1 + (r_a x d) I_a^-1 (r_a x d) + (r_b x d) I_b^-1 (r_b x d))
__device__ __forceinline__ float eff_mass(float ima, float imb, V3 rad, V3 iad, V3 rbd, V3 ibd) {
    const float den = ima + imb + dot(rad, iad) + dot(rbd, ibd);
    return den > 0.0f ? 1.0f / den : 0.0f;
}

__device__ __forceinline__ void build_row(Row &R, const DContact &c, const BodySm &B, int a, int b, float mu,
                                          float hs, float baumgarte) {
    const V3 n = ld3(c.n), xa = ld3(c.xa);
    const float phi = c.phi;
    const V3 xb = xa - phi * n;
    const V3 ra = xa - smv(B.com, a), rb = xb - smv(B.com, b);
    V3 t1, t2;
    tangent_basis(n, t1, t2);
    const V3 ran = cross(ra, n), rat1 = cross(ra, t1), rat2 = cross(ra, t2);
    const V3 rbn = cross(rb, n), rbt1 = cross(rb, t1), rbt2 = cross(rb, t2);
    const V3 ian = sym_mul(B.Iinv[a], ran), iat1 = sym_mul(B.Iinv[a], rat1), iat2 = sym_mul(B.Iinv[a], rat2);
    const V3 ibn = sym_mul(B.Iinv[b], rbn), ibt1 = sym_mul(B.Iinv[b], rbt1), ibt2 = sym_mul(B.Iinv[b], rbt2);
    st3(R.n, n); st3(R.t1, t1); st3(R.t2, t2);
    st3(R.ra_n, ran); st3(R.ra_t1, rat1); st3(R.ra_t2, rat2);
    st3(R.rb_n, rbn); st3(R.rb_t1, rbt1); st3(R.rb_t2, rbt2);
    st3(R.ia_n, ian); st3(R.ia_t1, iat1); st3(R.ia_t2, iat2);
    st3(R.ib_n, ibn); st3(R.ib_t1, ibt1); st3(R.ib_t2, ibt2);
    const float ima = B.invm[a], imb = B.invm[b];
    R.kn = eff_mass(ima, imb, ran, ian, rbn, ibn);
    R.kt1 = eff_mass(ima, imb, rat1, iat1, rbt1, ibt1);
    R.kt2 = eff_mass(ima, imb, rat2, iat2, rbt2, ibt2);
    R.bias = (phi > 0.0f) ? phi / hs : baumgarte * phi / hs;
    R.mu = mu;
    R.ln = 0.0f; R.lt1 = 0.0f; R.lt2 = 0.0f;
    R.a = a; R.b = b;
}

// One Gauss-Seidel sweep over the env's rows (lane 0 only).
__device__ void sweep(Row *rows, int nr, BodySm &B, bool use_bias) {
    for (int r = 0; r < nr; ++r) {
        Row &R = rows[r];
        if (R.kn == 0.0f) continue;
        const int a = R.a, b = R.b;
        V3 va = smv(B.v, a), wa = smv(B.w, a), vb = smv(B.v, b), wb = smv(B.w, b);
        const float ima = B.invm[a], imb = B.invm[b];
        // normal row
        const V3 n = ld3(R.n);
        float jv = dot(n, va - vb) + dot(ld3(R.ra_n), wa) - dot(ld3(R.rb_n), wb);
        if (use_bias) jv += R.bias;
        const float ln = fmaxf(R.ln - R.kn * jv, 0.0f);
        const float dl = ln - R.ln;
        R.ln = ln;
        va = va + (dl * ima) * n;
        wa = wa + dl * ld3(R.ia_n);
        vb = vb - (dl * imb) * n;
        wb = wb - dl * ld3(R.ib_n);
        // friction rows, projected jointly on the disk of radius mu lambda_n
        const V3 t1 = ld3(R.t1), t2 = ld3(R.t2);
        const V3 dv = va - vb;
        const float j1 = dot(t1, dv) + dot(ld3(R.ra_t1), wa) - dot(ld3(R.rb_t1), wb);
        const float j2 = dot(t2, dv) + dot(ld3(R.ra_t2), wa) - dot(ld3(R.rb_t2), wb);
        float l1 = R.lt1 - R.kt1 * j1, l2 = R.lt2 - R.kt2 * j2;
        const float lim = R.mu * ln;
        const float lt = sqrtf(l1 * l1 + l2 * l2);
        if (lt > lim) {
            const float s = lt > 0.0f ? lim / lt : 0.0f;
            l1 *= s;
            l2 *= s;
        }
        const float d1 = l1 - R.lt1, d2 = l2 - R.lt2;
        R.lt1 = l1;
        R.lt2 = l2;
        const V3 pt = d1 * t1 + d2 * t2;
        va = va + ima * pt;
        wa = wa + d1 * ld3(R.ia_t1) + d2 * ld3(R.ia_t2);
        vb = vb - imb * pt;
        wb = wb - (d1 * ld3(R.ib_t1) + d2 * ld3(R.ib_t2));
        smv_set(B.v, a, va); smv_set(B.w, a, wa);
        smv_set(B.v, b, vb); smv_set(B.w, b, wb);
    }
}

// Fast row of one contact, from the side of the movable body m (a or b of the pair):
//   f[0] = (d_n, k_n)        f[1] = (r x d_n, bias+e_n) f[2] = (I^-1 (r x d_n), mu)
//   f[3] = (d_1, k_t1)       f[4] = (r x d_1, e_1)      f[5] = (I^-1 (r x d_1), k_t2)
//   f[6] = (d_2, e_2)        f[7] = (r x d_2, e_n)      f[8] = (I^-1 (r x d_2), c_n1)
// and the row's impulse word (lambda_n, lambda_t1, lambda_t2, c_n2) in shared memory.
// d = s n, s t1, s t2 with s = +1 when m is body a (impulses +lambda d on m either way);
// e = -d . (v_o + w_o x r_o) is the partner's constant contribution to the row velocity;
// c_nk = ima d_k . d_n + (r x d_k) . I^-1 (r x d_n) is the change of friction row k's
// velocity per unit normal impulse of the same contact (an entry of J M^-1 J^T), so the
// friction rows need not wait for the velocity update of the normal row.
__device__ __forceinline__ void build_fast_row(float4 *f, float4 &lam0, const DContact &c, const BodySm &B, int a,
                                               int b, int m, float mu, float hs, float baumgarte) {
    lam0 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (m != a && m != b) {   // neither body of this pair can move: the contact does nothing
        for (int k = 0; k < kRowF4; ++k) f[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const bool ma = (m == a);
    const int o = ma ? b : a;
    const V3 n = ld3(c.n), xa = ld3(c.xa);
    const float phi = c.phi;
    const V3 xb = xa - phi * n;
    const V3 rm = (ma ? xa : xb) - smv(B.com, m);
    const V3 ro = (ma ? xb : xa) - smv(B.com, o);
    const float sg = ma ? 1.0f : -1.0f;
    V3 t1, t2;
    tangent_basis(n, t1, t2);
    const V3 dn = sg * n, d1 = sg * t1, d2 = sg * t2;
    const V3 uo = smv(B.v, o) + cross(smv(B.w, o), ro);
    const float ima = B.invm[m];
    const V3 rdn = cross(rm, dn), rd1 = cross(rm, d1), rd2 = cross(rm, d2);
    const V3 idn = sym_mul(B.Iinv[m], rdn), id1 = sym_mul(B.Iinv[m], rd1), id2 = sym_mul(B.Iinv[m], rd2);
    const float kn = eff_mass(ima, 0.0f, rdn, idn, v3(0, 0, 0), v3(0, 0, 0));
    const float kt1 = eff_mass(ima, 0.0f, rd1, id1, v3(0, 0, 0), v3(0, 0, 0));
    const float kt2 = eff_mass(ima, 0.0f, rd2, id2, v3(0, 0, 0), v3(0, 0, 0));
    const float bias = (phi > 0.0f) ? phi / hs : baumgarte * phi / hs;
    if (kn == 0.0f) {   // the movable body cannot respond along n: the contact does nothing
        for (int k = 0; k < kRowF4; ++k) f[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    f[0] = make_float4(dn.x, dn.y, dn.z, kn);
    f[1] = make_float4(rdn.x, rdn.y, rdn.z, bias - dot(dn, uo));
    f[2] = make_float4(idn.x, idn.y, idn.z, mu);
    f[3] = make_float4(d1.x, d1.y, d1.z, kt1);
    f[4] = make_float4(rd1.x, rd1.y, rd1.z, -dot(d1, uo));
    f[5] = make_float4(id1.x, id1.y, id1.z, kt2);
    f[6] = make_float4(d2.x, d2.y, d2.z, -dot(d2, uo));
    f[7] = make_float4(rd2.x, rd2.y, rd2.z, -dot(dn, uo));
    f[8] = make_float4(id2.x, id2.y, id2.z, ima * dot(d1, dn) + dot(rd1, idn));
    lam0.w = ima * dot(d2, dn) + dot(rd2, idn);
}

// `passes` Gauss-Seidel sweeps over nr fast rows by one group of G lanes (one env),
// kRowBlock rows at a time.  All lanes of the warp run the same number of blocks (enough
// for the largest total of its groups; rows past a group's own total are computed and
// discarded), so every __syncwarp is reached by the whole warp.  Lanes of a group hold
// identical values.  Per block: wait for its rows' copy group, read the rows and their
// impulse words into registers, let the group's lanes refill those ring slots with the
// rows kRing positions ahead (one cp.async per float4, one commit group per block), then
// solve the rows with no barrier in between, so the compiler can overlap one row's
// velocity update with the next row's independent work.  Lane 0 of the group stores the
// impulses; the next block's __syncwarp orders those stores before any later read.  An
// impulse word read for a row that repeats inside the block (nr smaller than the block)
// is replaced by the value just computed.  A row written all-zero (a contact neither body
// can act on) leaves every value unchanged.
__device__ __forceinline__ void ring_read(const float4 *sp, float4 (&f)[kRowF4]) {
#pragma unroll
    for (int k = 0; k < kRowF4; ++k) f[k] = sp[k];
}

template <int G>
__device__ __forceinline__ void ring_fill(float4 *ring, int slot, const float4 *rows, int pf, int nr, int gl) {
    if (nr > 0) {
#pragma unroll
        for (int k = gl; k < kRowF4; k += G) cp_async16(ring + kRowF4 * slot + k, rows + kRowF4 * pf + k);
    }
}

template <int G, bool kBias>
__device__ void sweep_fast(const float4 *rows, int nr, int total, int trips, float4 *ring, float4 *lam, V3 &va,
                           V3 &wa, float ima, int gl) {
    constexpr int RB = kRowBlock;
    if (trips == 0) return;   // warp-uniform
    int r = 0, pf = 0;
    for (int s = 0; s < kRing; s += RB) {
#pragma unroll
        for (int b = 0; b < RB; ++b) {
            ring_fill<G>(ring, s + b, rows, pf, nr, gl);
            if (++pf >= nr) pf = 0;
        }
        cp_async_commit();
    }
    for (int q0 = 0; q0 < trips; q0 += RB) {
        const int slot0 = q0 & (kRing - 1);
        asm volatile("cp.async.wait_group %0;\n" ::"n"(kRing / RB - 1) : "memory");
        __syncwarp();
        float4 f[RB][kRowF4], L[RB];
        int rr[RB];
#pragma unroll
        for (int b = 0; b < RB; ++b) {
            ring_read(ring + kRowF4 * (slot0 + b), f[b]);
            rr[b] = r;
            L[b] = lam[r];
            if (++r >= nr) r = 0;
        }
        __syncwarp();
#pragma unroll
        for (int b = 0; b < RB; ++b) {
            ring_fill<G>(ring, slot0 + b, rows, pf, nr, gl);
            if (++pf >= nr) pf = 0;
        }
        cp_async_commit();
        float4 nl[RB];
#pragma unroll
        for (int b = 0; b < RB; ++b) {
            float4 Lb = L[b];
#pragma unroll
            for (int bp = 0; bp < b; ++bp)
                if (b - bp == nr) Lb = nl[bp];   // this row already ran in the block
            const float4 *F = f[b];
            const float jv = __fmaf_rn(F[0].z, va.z, __fmaf_rn(F[0].y, va.y, __fmaf_rn(F[0].x, va.x, kBias ? F[1].w : F[7].w))) +
                             __fmaf_rn(F[1].z, wa.z, __fmaf_rn(F[1].y, wa.y, F[1].x * wa.x));
            const float j1b = __fmaf_rn(F[3].z, va.z, __fmaf_rn(F[3].y, va.y, __fmaf_rn(F[3].x, va.x, F[4].w))) +
                              __fmaf_rn(F[4].z, wa.z, __fmaf_rn(F[4].y, wa.y, F[4].x * wa.x));
            const float j2b = __fmaf_rn(F[6].z, va.z, __fmaf_rn(F[6].y, va.y, __fmaf_rn(F[6].x, va.x, F[6].w))) +
                              __fmaf_rn(F[7].z, wa.z, __fmaf_rn(F[7].y, wa.y, F[7].x * wa.x));
            // normal row
            const float ln = fmaxf(__fmaf_rn(-F[0].w, jv, Lb.x), 0.0f);
            float dl = ln - Lb.x;
            // friction rows after the normal change, projected jointly on |lambda_t| <= mu lambda_n
            const float t1 = __fmaf_rn(-F[3].w, __fmaf_rn(dl, F[8].w, j1b), Lb.y);
            const float t2 = __fmaf_rn(-F[5].w, __fmaf_rn(dl, Lb.w, j2b), Lb.z);
            const float sc = fminf(1.0f, (F[2].w * ln) * rsqrtf(__fmaf_rn(t1, t1, t2 * t2)));
            const float l1 = t1 * sc, l2 = t2 * sc;
            float e1 = l1 - Lb.y, e2 = l2 - Lb.z;
            nl[b] = make_float4(ln, l1, l2, Lb.w);
            const bool act = q0 + b < total;
            if (!act) { dl = 0.0f; e1 = 0.0f; e2 = 0.0f; }
            if (act && gl == 0) lam[rr[b]] = nl[b];
            const float dlm = dl * ima, e1m = e1 * ima, e2m = e2 * ima;
            va = v3(__fmaf_rn(e2m, F[6].x, __fmaf_rn(e1m, F[3].x, __fmaf_rn(dlm, F[0].x, va.x))),
                    __fmaf_rn(e2m, F[6].y, __fmaf_rn(e1m, F[3].y, __fmaf_rn(dlm, F[0].y, va.y))),
                    __fmaf_rn(e2m, F[6].z, __fmaf_rn(e1m, F[3].z, __fmaf_rn(dlm, F[0].z, va.z))));
            wa = v3(__fmaf_rn(e2, F[8].x, __fmaf_rn(e1, F[5].x, __fmaf_rn(dl, F[2].x, wa.x))),
                    __fmaf_rn(e2, F[8].y, __fmaf_rn(e1, F[5].y, __fmaf_rn(dl, F[2].y, wa.y))),
                    __fmaf_rn(e2, F[8].z, __fmaf_rn(e1, F[5].z, __fmaf_rn(dl, F[2].z, wa.z))));
        }
    }
    cp_async_wait_all();
    __syncwarp();
}


template <int G>
__device__ __forceinline__ int warp_max(int v) {
#pragma unroll
    for (int off = G; off < 32; off <<= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}

// One substep's solve for kGroups envs per warp (G = 32 / kGroups lanes each) and
// blockDim.x / 32 warps per block.  No block-wide barrier: every warp is independent.
template <int kGroups>
__global__ void __launch_bounds__(kSolveMaxWarps * 32) solve_kernel(SimParams p) {
    constexpr int G = 32 / kGroups;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane / G, gl = lane % G;
    const int per_block = (blockDim.x >> 5) * kGroups;
    const int slot = warp * kGroups + grp;
    const int e0 = blockIdx.x * per_block + warp * kGroups;
    if (e0 >= p.n_envs) return;   // the whole warp has no env
    const int e = e0 + grp;
    const bool valid = e < p.n_envs;
    EnvDev E;
    if (valid) {
        E = p.envs[e];
    } else {
        E.first_body = 0; E.n_bodies = 0; E.first_pair = 0; E.n_pairs = 0;
        E.row_off = 0; E.row_cap = 0; E.movable = -1;
    }
    extern __shared__ __align__(16) float4 dyn_smem[];
    float4 *env_base = dyn_smem + (size_t)slot * env_stride_f4(p.lam_cap);
    __shared__ EnvSm S_all[kSolveMaxWarps * kGroups];
    EnvSm &S = S_all[slot];
    BodySm &B = S.B;
    const float hs = p.hs;
    // 1. external forces; world inertia at the substep's start
    for (int lb = gl; lb < E.n_bodies; lb += G) {
        const int bi = E.first_body + lb;
        const BodyProps P = p.props[bi];
        const float4 q = make_float4(p.quat[4 * bi], p.quat[4 * bi + 1], p.quat[4 * bi + 2], p.quat[4 * bi + 3]);
        const M3 R = quat_to_mat(q);
        V3 pos = ld3(p.pos + 3 * bi), v = ld3(p.linvel + 3 * bi), w = ld3(p.angvel + 3 * bi);
        const V3 com = mul(R, ld3(P.com_b)) + pos;
        float Iw[6], Ii[6] = {0, 0, 0, 0, 0, 0};
        rot_sym(R, P.Ib, Iw);
        if (P.type == FW_BODY_DYNAMIC) {
            rot_sym(R, P.Ib_inv, Ii);
            const V3 gv = v3(p.gravity[0], p.gravity[1], p.gravity[2]);
            v = v + hs * (gv + P.invm * ld3(P.force));
            const V3 tau = ld3(P.torque) - cross(w, sym_mul(Iw, w));
            w = w + hs * sym_mul(Ii, tau);
        } else if (P.type == FW_BODY_FIXED_AXIS) {
            const V3 ax = ld3(P.axis);
            const float Iaa = dot(ax, sym_mul(Iw, ax));
            const float s = 1.0f / Iaa;
            Ii[0] = ax.x * ax.x * s; Ii[1] = ax.y * ax.y * s; Ii[2] = ax.z * ax.z * s;
            Ii[3] = ax.x * ax.y * s; Ii[4] = ax.x * ax.z * s; Ii[5] = ax.y * ax.z * s;
            w = w + (hs * dot(ax, ld3(P.torque)) * s) * ax;
        }
        smv_set(B.v, lb, v);
        smv_set(B.w, lb, w);
        smv_set(B.com, lb, com);
        B.invm[lb] = P.invm;
        for (int k = 0; k < 6; ++k) B.Iinv[lb][k] = Ii[k];
    }
    // row offsets of the env's pairs
    if (gl == 0) {
        int acc = 0;
        for (int k = 0; k < E.n_pairs; ++k) {
            S.row_base[k] = acc;
            const int c = p.counts[E.first_pair + k];
            acc += c < p.cap_pair ? c : p.cap_pair;
        }
        S.row_base[E.n_pairs] = acc;
    }
    __syncwarp();
    const int nr = S.row_base[E.n_pairs];
    Row *rows = p.rows + E.row_off;
    float4 *lam = env_base;
    float4 *ring = lam + p.lam_cap;
    const int m = E.movable;
    const bool fast = (m != -2) && nr <= p.lam_cap;
    float4 *frows = reinterpret_cast<float4 *>(rows);
    // 2. constraint preparation, one contact per lane, then the couplings between neighbours
    for (int k = 0; k < E.n_pairs; ++k) {
        const int pi = E.first_pair + k;
        const PairDev P = p.pairs[pi];
        const int cnt = S.row_base[k + 1] - S.row_base[k];
        for (int i = gl; i < cnt; i += G) {
            const DContact &c = p.contacts[(long long)pi * p.cap_pair + i];
            if (fast) {
                if (m >= 0)
                    build_fast_row(frows + kRowF4 * (S.row_base[k] + i), lam[S.row_base[k] + i], c, B, P.local_a,
                                   P.local_b, m, P.mu, hs, p.baumgarte);
            } else {
                build_row(rows[S.row_base[k] + i], c, B, P.local_a, P.local_b, P.mu, hs, p.baumgarte);
            }
        }
    }
    __threadfence_block();
    __syncwarp();
    // 3. Gauss-Seidel sweeps (no movable body: nothing to solve)
    const bool run_fast = valid && fast && m >= 0;
    {
        const int total = run_fast ? nr * p.n_iters : 0;
        const int trips = warp_max<G>(total);
        V3 va = v3(0, 0, 0), wa = v3(0, 0, 0);
        float ima = 0.0f;
        if (run_fast) { va = smv(B.v, m); wa = smv(B.w, m); ima = B.invm[m]; }
        sweep_fast<G, true>(frows, run_fast ? nr : 0, total, trips, ring, lam, va, wa, ima, gl);
        if (run_fast && gl == 0) { smv_set(B.v, m, va); smv_set(B.w, m, wa); }
    }
    if (valid && !fast && gl == 0) {
        for (int it = 0; it < p.n_iters; ++it) sweep(rows, nr, B, true);
    }
    __syncwarp();
    // 4. integration
    for (int lb = gl; lb < E.n_bodies; lb += G) {
        const int bi = E.first_body + lb;
        const BodyProps P = p.props[bi];
        if (P.type != FW_BODY_STATIC) {
            V3 w = smv(B.w, lb);
            const V3 v = smv(B.v, lb);
            if ((P.type == FW_BODY_DYNAMIC || P.type == FW_BODY_FIXED_AXIS) && p.max_angvel > 0.0f) {
                const float wn = sqrtf(dot(w, w));
                if (wn > p.max_angvel) w = (p.max_angvel / wn) * w;
                smv_set(B.w, lb, w);
            }
            const V3 com = smv(B.com, lb) + hs * v;
            float4 q = make_float4(p.quat[4 * bi], p.quat[4 * bi + 1], p.quat[4 * bi + 2], p.quat[4 * bi + 3]);
            // dq = (omega, 0) (x) q
            const float dx = q.w * w.x + w.y * q.z - w.z * q.y;
            const float dy = q.w * w.y + w.z * q.x - w.x * q.z;
            const float dz = q.w * w.z + w.x * q.y - w.y * q.x;
            const float dw = -(w.x * q.x + w.y * q.y + w.z * q.z);
            const float hh = 0.5f * hs;
            q.x += hh * dx; q.y += hh * dy; q.z += hh * dz; q.w += hh * dw;
            const float inv = 1.0f / sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
            q.x *= inv; q.y *= inv; q.z *= inv; q.w *= inv;
            const M3 R = quat_to_mat(q);
            const V3 pos = com - mul(R, ld3(P.com_b));
            st3(p.pos + 3 * bi, pos);
            S.q_new[lb][0] = q.x; S.q_new[lb][1] = q.y; S.q_new[lb][2] = q.z; S.q_new[lb][3] = q.w;
            const bool bad = !(isfinite(pos.x) && isfinite(pos.y) && isfinite(pos.z) && isfinite(q.x) &&
                               isfinite(q.y) && isfinite(q.z) && isfinite(q.w));
            if (bad) atomicOr(p.status, kStatusNonFinite);
        } else {
            for (int k = 0; k < 4; ++k) S.q_new[lb][k] = p.quat[4 * bi + k];
        }
    }
    __syncwarp();
    // 5. optional bias-free sweeps
    if (p.n_vel_iters > 0) {
        const int total = run_fast ? nr * p.n_vel_iters : 0;
        const int trips = warp_max<G>(total);
        V3 va = v3(0, 0, 0), wa = v3(0, 0, 0);
        float ima = 0.0f;
        if (run_fast) { va = smv(B.v, m); wa = smv(B.w, m); ima = B.invm[m]; }
        sweep_fast<G, false>(frows, run_fast ? nr : 0, total, trips, ring, lam, va, wa, ima, gl);
        if (run_fast && gl == 0) { smv_set(B.v, m, va); smv_set(B.w, m, wa); }
        if (valid && !fast && gl == 0) {
            for (int it = 0; it < p.n_vel_iters; ++it) sweep(rows, nr, B, false);
        }
    }
    __syncwarp();
    for (int lb = gl; lb < E.n_bodies; lb += G) {
        const int bi = E.first_body + lb;
        for (int k = 0; k < 4; ++k) p.quat[4 * bi + k] = S.q_new[lb][k];
        const V3 v = smv(B.v, lb), w = smv(B.w, lb);
        st3(p.linvel + 3 * bi, v);
        st3(p.angvel + 3 * bi, w);
        if (!(isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(w.x) && isfinite(w.y) && isfinite(w.z)))
            atomicOr(p.status, kStatusNonFinite);
    }
}

__global__ void normalize_quats_kernel(float *q, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float x = q[4 * i], y = q[4 * i + 1], z = q[4 * i + 2], w = q[4 * i + 3];
    const float inv = 1.0f / sqrtf(x * x + y * y + z * z + w * w);
    q[4 * i] = x * inv; q[4 * i + 1] = y * inv; q[4 * i + 2] = z * inv; q[4 * i + 3] = w * inv;
}

}  // namespace

cudaError_t launch_normalize_quats(float *quat, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    normalize_quats_kernel<<<(n + 255) / 256, 256, 0, s>>>(quat, n);
    return cudaGetLastError();
}

size_t solve_smem_bytes(int lam_cap) { return sizeof(float4) * (size_t)env_stride_f4(lam_cap); }

template <int kGroups>
static cudaError_t prepare_one(int optin, int *max_dyn) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, solve_kernel<kGroups>);
    if (e != cudaSuccess) return e;
    *max_dyn = optin - (int)a.sharedSizeBytes;
    return cudaFuncSetAttribute(solve_kernel<kGroups>, cudaFuncAttributeMaxDynamicSharedMemorySize, *max_dyn);
}

cudaError_t prepare_solve(int optin, int max_dyn[4]) {
    cudaError_t e = prepare_one<1>(optin, &max_dyn[0]);
    if (e == cudaSuccess) e = prepare_one<2>(optin, &max_dyn[1]);
    if (e == cudaSuccess) e = prepare_one<4>(optin, &max_dyn[2]);
    if (e == cudaSuccess) e = prepare_one<8>(optin, &max_dyn[3]);
    return e;
}

SolveShape solve_shape(int n_envs, int lam_cap, int groups, int warps, const int max_dyn[4], int n_sm) {
    const size_t per_env = solve_smem_bytes(lam_cap);
    auto cap = [&](int g) { return (size_t)max_dyn[g == 1 ? 0 : g == 2 ? 1 : g == 4 ? 2 : 3]; };
    if (groups != 1 && groups != 2 && groups != 4 && groups != 8) groups = 0;
    const int sms = n_sm > 0 ? n_sm : 1;
    if (groups == 0) {   // at most one warp per scheduler (4 per SM); two envs per warp at least,
                         // which measured faster than one per warp even with warps to spare
        const int want = (n_envs + 4 * sms - 1) / (4 * sms);
        groups = want <= 2 ? 2 : (want <= 4 ? 4 : 8);
    }
    while (groups > 1 && per_env * groups > cap(groups)) groups >>= 1;
    if (warps < 1 || warps > kSolveMaxWarps) {   // spread the warps over every SM first
        const int n_warps = (n_envs + groups - 1) / groups;
        warps = (n_warps + sms - 1) / sms;
        warps = warps < 1 ? 1 : (warps > kSolveMaxWarps ? kSolveMaxWarps : warps);
    }
    while (warps > 1 && per_env * groups * warps > cap(groups)) --warps;
    SolveShape sh;
    sh.groups = groups;
    sh.warps = warps;
    sh.smem = per_env * groups * warps;
    return sh;
}

cudaError_t launch_solve(const SimParams &p, const SolveShape &sh, cudaStream_t s) {
    if (p.n_envs == 0) return cudaSuccess;
    const int per_block = sh.groups * sh.warps;
    const int blocks = (p.n_envs + per_block - 1) / per_block;
    if (sh.groups == 1) solve_kernel<1><<<blocks, 32 * sh.warps, sh.smem, s>>>(p);
    else if (sh.groups == 2) solve_kernel<2><<<blocks, 32 * sh.warps, sh.smem, s>>>(p);
    else if (sh.groups == 4) solve_kernel<4><<<blocks, 32 * sh.warps, sh.smem, s>>>(p);
    else solve_kernel<8><<<blocks, 32 * sh.warps, sh.smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace fw
