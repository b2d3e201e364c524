// fw_solve.cu -- contact solution of one substep (Sec. III-B): external forces,
// constraint preparation, Gauss-Seidel sweeps with Coulomb friction, integration.
// One warp per environment: lanes prepare rows and integrate bodies in parallel; the
// sweep itself is the serial Gauss-Seidel chain and runs on lane 0.
//
// Two sweep forms compute the same update.  Fast form (an env with at most one movable
// body, i.e. every other body static or kinematic): each contact is written from the
// movable body's side (directions negated when it is the pair's SDF body, the partner's
// prescribed velocity folded into a constant), 9 float4 per contact; the body's velocity
// stays in registers, the rows stream from global memory through a cp.async ring in
// shared memory and the accumulated impulses live in shared memory.  General form
// (several movable bodies): full two-body rows, velocities in shared memory.
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

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_ring() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(kRing - 1) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

struct BodySm {
    float v[kMaxBodies][3], w[kMaxBodies][3];
    float invm[kMaxBodies];
    float Iinv[kMaxBodies][6];
    float com[kMaxBodies][3];
};

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
//   f[6] = (d_2, e_2)        f[7] = (r x d_2, e_n)      f[8] = (I^-1 (r x d_2), 0)
// d = s n, s t1, s t2 with s = +1 when m is body a (impulses +lambda d on m either way);
// e = -d . (v_o + w_o x r_o) is the partner's constant contribution to the row velocity.
__device__ __forceinline__ void build_fast_row(float4 *f, const DContact &c, const BodySm &B, int a, int b, int m,
                                               float mu, float hs, float baumgarte) {
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
    f[8] = make_float4(id2.x, id2.y, id2.z, 0.0f);
}

// `passes` Gauss-Seidel sweeps over nr fast rows.  The whole warp runs the loop with
// identical values in every lane (uniform control flow); lanes 0..8 copy one float4 each
// of the row kRing positions ahead into the ring with one cp.async instruction, and lane
// 0 stores the impulses.  One commit group per row keeps "row q has landed" equal to "at
// most kRing - 1 groups pending"; __syncwarp makes a landed row visible to all lanes and
// orders the reads of a slot before its refill.  Row q+1 is read into registers while
// row q is solved, so the shared-memory latency stays off the Gauss-Seidel chain.  A row
// written all-zero (a contact neither body can act on) leaves every value unchanged.
__device__ __forceinline__ void ring_read(const float4 *sp, float4 f[kRowF4]) {
#pragma unroll
    for (int k = 0; k < kRowF4; ++k) f[k] = sp[k];
}

// One row of the fast sweep: solves the row held in f while the next row (slot nslot)
// is read into g.
struct SweepState {
    V3 va, wa;
    int r, slot, pf;
};

__device__ __forceinline__ void sweep_row(const float4 (&f)[kRowF4], float4 (&g)[kRowF4], SweepState &st,
                                          const float4 *rows, int nr, float4 *ring, float4 *lam, float ima,
                                          bool use_bias, int lane) {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(kRing - 2) : "memory");
    __syncwarp();
    const int nslot = (st.slot + 1) & (kRing - 1);
    ring_read(ring + kRowF4 * nslot, g);
    const float4 L = lam[st.r];
    V3 va = st.va, wa = st.wa;
    // normal row: two independent three-term chains
    float jv = (f[0].x * va.x + f[0].y * va.y + f[0].z * va.z) + (f[1].x * wa.x + f[1].y * wa.y + f[1].z * wa.z);
    jv += use_bias ? f[1].w : f[7].w;
    const float ln = fmaxf(__fmaf_rn(-f[0].w, jv, L.x), 0.0f);
    const float dl = ln - L.x;
    const float dlm = dl * ima;
    va = v3(__fmaf_rn(dlm, f[0].x, va.x), __fmaf_rn(dlm, f[0].y, va.y), __fmaf_rn(dlm, f[0].z, va.z));
    wa = v3(__fmaf_rn(dl, f[2].x, wa.x), __fmaf_rn(dl, f[2].y, wa.y), __fmaf_rn(dl, f[2].z, wa.z));
    // friction rows, projected jointly on the disk of radius mu lambda_n
    const float j1 = (f[3].x * va.x + f[3].y * va.y + f[3].z * va.z) + (f[4].x * wa.x + f[4].y * wa.y + f[4].z * wa.z) + f[4].w;
    const float j2 = (f[6].x * va.x + f[6].y * va.y + f[6].z * va.z) + (f[7].x * wa.x + f[7].y * wa.y + f[7].z * wa.z) + f[6].w;
    const float t1 = __fmaf_rn(-f[3].w, j1, L.y), t2 = __fmaf_rn(-f[5].w, j2, L.z);
    const float lim = f[2].w * ln;
    const float lt2 = t1 * t1 + t2 * t2;
    const float sc = (lt2 > lim * lim) ? lim * rsqrtf(lt2) : 1.0f;
    const float l1 = t1 * sc, l2 = t2 * sc;
    const float e1 = l1 - L.y, e2 = l2 - L.z;
    const float e1m = e1 * ima, e2m = e2 * ima;
    st.va = v3(__fmaf_rn(e2m, f[6].x, __fmaf_rn(e1m, f[3].x, va.x)), __fmaf_rn(e2m, f[6].y, __fmaf_rn(e1m, f[3].y, va.y)),
               __fmaf_rn(e2m, f[6].z, __fmaf_rn(e1m, f[3].z, va.z)));
    st.wa = v3(__fmaf_rn(e2, f[8].x, __fmaf_rn(e1, f[5].x, wa.x)), __fmaf_rn(e2, f[8].y, __fmaf_rn(e1, f[5].y, wa.y)),
               __fmaf_rn(e2, f[8].z, __fmaf_rn(e1, f[5].z, wa.z)));
    if (lane == 0) lam[st.r] = make_float4(ln, l1, l2, 0.0f);
    __syncwarp();
    // refill this slot with the row kRing positions ahead (past the end: an unused copy)
    if (lane < kRowF4) cp_async16(ring + kRowF4 * st.slot + lane, rows + kRowF4 * st.pf + lane);
    cp_async_commit();
    if (++st.pf == nr) st.pf = 0;
    if (++st.r == nr) st.r = 0;
    st.slot = nslot;
}

__device__ void sweep_fast(const float4 *rows, int nr, int passes, float4 *ring, float4 *lam, V3 &va, V3 &wa,
                           float ima, bool use_bias) {
    const int lane = threadIdx.x & 31;
    const int total = nr * passes;
    if (total == 0) return;
    SweepState st;
    st.va = va; st.wa = wa; st.r = 0; st.slot = 0; st.pf = 0;
    for (int q = 0; q < kRing; ++q) {
        if (lane < kRowF4) cp_async16(ring + kRowF4 * q + lane, rows + kRowF4 * st.pf + lane);
        cp_async_commit();
        if (++st.pf == nr) st.pf = 0;
    }
    float4 f[kRowF4], g[kRowF4];
    cp_async_wait_ring();
    __syncwarp();
    ring_read(ring, f);
    int q = 0;
    for (; q + 1 < total; q += 2) {   // two rows per trip, the register sets trade roles
        sweep_row(f, g, st, rows, nr, ring, lam, ima, use_bias, lane);
        sweep_row(g, f, st, rows, nr, ring, lam, ima, use_bias, lane);
    }
    if (q < total) sweep_row(f, g, st, rows, nr, ring, lam, ima, use_bias, lane);
    va = st.va;
    wa = st.wa;
    cp_async_wait_all();
    __syncwarp();
}

__global__ void __launch_bounds__(32) solve_kernel(SimParams p) {
    const int e = blockIdx.x;
    const int lane = threadIdx.x;
    const EnvDev E = p.envs[e];
    __shared__ BodySm B;
    __shared__ float q_new[kMaxBodies][4];
    __shared__ int row_base[64];
    const float hs = p.hs;
    // 1. external forces; world inertia at the substep's start
    if (lane < E.n_bodies) {
        const int bi = E.first_body + lane;
        const BodyProps P = p.props[bi];
        const float4 q = make_float4(p.quat[4 * bi], p.quat[4 * bi + 1], p.quat[4 * bi + 2], p.quat[4 * bi + 3]);
        const M3 R = quat_to_mat(q);
        V3 pos = ld3(p.pos + 3 * bi), v = ld3(p.linvel + 3 * bi), w = ld3(p.angvel + 3 * bi);
        const V3 com = mul(R, ld3(P.com_b)) + pos;
        float Iw[6], Ii[6] = {0, 0, 0, 0, 0, 0};
        rot_sym(R, P.Ib, Iw);
        if (P.type == FW_BODY_DYNAMIC) {
            rot_sym(R, P.Ib_inv, Ii);
            const V3 g = v3(p.gravity[0], p.gravity[1], p.gravity[2]);
            v = v + hs * (g + P.invm * ld3(P.force));
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
        smv_set(B.v, lane, v);
        smv_set(B.w, lane, w);
        smv_set(B.com, lane, com);
        B.invm[lane] = P.invm;
        for (int k = 0; k < 6; ++k) B.Iinv[lane][k] = Ii[k];
    }
    // row offsets of the env's pairs
    if (lane == 0) {
        int acc = 0;
        for (int k = 0; k < E.n_pairs; ++k) {
            row_base[k] = acc;
            const int c = p.counts[E.first_pair + k];
            acc += c < p.cap_pair ? c : p.cap_pair;
        }
        row_base[E.n_pairs] = acc;
    }
    __syncwarp();
    const int nr = row_base[E.n_pairs];
    Row *rows = p.rows + E.row_off;
    extern __shared__ __align__(16) float4 dyn_smem[];
    const int m = E.movable;
    const bool fast = (m != -2) && nr <= p.lam_cap;
    float4 *frows = reinterpret_cast<float4 *>(rows);
    float4 *lam = dyn_smem;
    float4 *ring = dyn_smem + p.lam_cap;
    // 2. constraint preparation, one contact per lane
    for (int k = 0; k < E.n_pairs; ++k) {
        const int pi = E.first_pair + k;
        const PairDev P = p.pairs[pi];
        const int cnt = row_base[k + 1] - row_base[k];
        for (int i = lane; i < cnt; i += 32) {
            const DContact &c = p.contacts[(long long)pi * p.cap_pair + i];
            if (fast) {
                if (m >= 0) {
                    build_fast_row(frows + kRowF4 * (row_base[k] + i), c, B, P.local_a, P.local_b, m, P.mu, hs,
                                   p.baumgarte);
                    lam[row_base[k] + i] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            } else {
                build_row(rows[row_base[k] + i], c, B, P.local_a, P.local_b, P.mu, hs, p.baumgarte);
            }
        }
    }
    __threadfence_block();
    __syncwarp();
    // 3. Gauss-Seidel sweeps (no movable body: nothing to solve)
    if (fast) {
        if (m >= 0) {
            V3 va = smv(B.v, m), wa = smv(B.w, m);
            sweep_fast(frows, nr, p.n_iters, ring, lam, va, wa, B.invm[m], true);
            if (lane == 0) { smv_set(B.v, m, va); smv_set(B.w, m, wa); }
        }
    } else if (lane == 0) {
        for (int it = 0; it < p.n_iters; ++it) sweep(rows, nr, B, true);
    }
    __syncwarp();
    // 4. integration
    if (lane < E.n_bodies) {
        const int bi = E.first_body + lane;
        const BodyProps P = p.props[bi];
        if (P.type != FW_BODY_STATIC) {
            V3 w = smv(B.w, lane);
            const V3 v = smv(B.v, lane);
            if ((P.type == FW_BODY_DYNAMIC || P.type == FW_BODY_FIXED_AXIS) && p.max_angvel > 0.0f) {
                const float wn = sqrtf(dot(w, w));
                if (wn > p.max_angvel) w = (p.max_angvel / wn) * w;
                smv_set(B.w, lane, w);
            }
            const V3 com = smv(B.com, lane) + hs * v;
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
            q_new[lane][0] = q.x; q_new[lane][1] = q.y; q_new[lane][2] = q.z; q_new[lane][3] = q.w;
            const bool bad = !(isfinite(pos.x) && isfinite(pos.y) && isfinite(pos.z) && isfinite(q.x) &&
                               isfinite(q.y) && isfinite(q.z) && isfinite(q.w));
            if (bad) atomicOr(p.status, kStatusNonFinite);
        } else {
            for (int k = 0; k < 4; ++k) q_new[lane][k] = p.quat[4 * bi + k];
        }
    }
    __syncwarp();
    // 5. optional bias-free sweeps
    if (p.n_vel_iters > 0) {
        if (fast) {
            if (m >= 0) {
                V3 va = smv(B.v, m), wa = smv(B.w, m);
                sweep_fast(frows, nr, p.n_vel_iters, ring, lam, va, wa, B.invm[m], false);
                if (lane == 0) { smv_set(B.v, m, va); smv_set(B.w, m, wa); }
            }
        } else if (lane == 0) {
            for (int it = 0; it < p.n_vel_iters; ++it) sweep(rows, nr, B, false);
        }
    }
    __syncwarp();
    if (lane < E.n_bodies) {
        const int bi = E.first_body + lane;
        for (int k = 0; k < 4; ++k) p.quat[4 * bi + k] = q_new[lane][k];
        const V3 v = smv(B.v, lane), w = smv(B.w, lane);
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

size_t solve_smem_bytes(int lam_cap) { return sizeof(float4) * ((size_t)lam_cap + (size_t)kRing * kRowF4); }

cudaError_t prepare_solve(int max_lam_cap) {
    return cudaFuncSetAttribute(solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)solve_smem_bytes(max_lam_cap));
}

cudaError_t launch_solve(const SimParams &p, cudaStream_t s) {
    if (p.n_envs == 0) return cudaSuccess;
    solve_kernel<<<p.n_envs, 32, solve_smem_bytes(p.lam_cap), s>>>(p);
    return cudaGetLastError();
}

}  // namespace fw
