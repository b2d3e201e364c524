// fw_solve.cu -- contact solution of one substep (Sec. III-B): external forces,
// constraint preparation, Gauss-Seidel sweeps with Coulomb friction, integration.
// A group of lanes per environment (a whole warp, or 16, 8 or 4 lanes when several envs
// share a warp): its lanes prepare rows and integrate bodies in parallel; the sweep itself is
// the serial Gauss-Seidel chain, run with identical values by every lane of the group.
//
// Two sweep forms compute the same update.  Fast form (an env with at most one movable
// body, i.e. every other body static or kinematic): each contact is written from the
// movable body's side (directions negated when it is the pair's SDF body, the partner's
// prescribed velocity folded into a constant), 15 float4 per contact; the body's velocity
// stays in registers, split between the group's even lanes (linear part) and odd lanes
// (angular part), the rows stream from global memory into shared memory in chunks of 16
// rows, one cp.async.bulk copy per chunk issued by one lane and completed on an mbarrier
// (two chunk buffers: the next chunk is in flight while one is read), and the accumulated
// impulses live in shared memory.  General form
// (several movable bodies): full two-body rows streamed through the same ring by one lane,
// impulses and velocities in shared memory.
//
// Update rule (velocity-level projected Gauss-Seidel; the paper cites the solver without
// restating it): per contact, the normal row
//     lambda_n <- max(0, lambda_n - k_n (n . v_rel + b)),
// then both friction rows from the updated velocities, lambda_t <- lambda_t - k_t (t . v_rel),
// projected jointly on the disk |lambda_t| <= mu lambda_n; every change is applied to
// both bodies at once.  b = phi/hs for phi > 0 (speculative contact), baumgarte*phi/hs
// otherwise.  Integration: semi-implicit Euler of the centre of mass and
// q <- normalize(q + hs/2 (omega, 0) q).
//
// The weighted Jacobi solver (solver = 1, sweep_jacobi) is the alternative the paper's
// solver comparison sizes: per sweep every contact's block update from the sweep-start
// velocity, all taken with the weight 1 / (contacts that can act); it runs on fast rows,
// an env's contacts in parallel on its lanes.
#include "fw_device.cuh"

namespace fw {

namespace {

constexpr int kMaxBodies = 8;
constexpr int kRing = 16;     // rows in flight in the general form's shared-memory ring
constexpr int kRowF4 = 15;    // float4 per fast row
constexpr int kHalfF4 = 6;    // float4 of a row's linear (even lanes) or angular (odd lanes) half
static_assert(kChunk * kRowF4 * 16 % 16 == 0, "bulk copies move multiples of 16 bytes");
constexpr int kChunkF4 = kChunk * kRowF4;                  // one chunk of rows: 240 float4, 3840 bytes
constexpr unsigned kChunkBytes = kChunkF4 * 16;
constexpr int kChunkBufs = 2;                              // chunk buffers per env
constexpr int kBarF4 = 1;                                  // their 2 mbarriers (8 bytes each)
constexpr int kSlotF4 = kChunkBufs * kChunkF4 + kBarF4;    // per env beside its impulse words
static_assert(kSlotF4 >= kRing * kRowF4 + kBarF4, "the general form's ring fits in the chunk buffers");
constexpr int kWaitTries = 1 << 20;                        // bounded mbarrier waits

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// ---- mbarriers and bulk copies (the fast sweep's chunked row stream)
__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
// makes this thread's global writes (the rows) visible to later bulk copies (async proxy)
__device__ __forceinline__ void fence_async_global() { asm volatile("fence.proxy.async.global;\n" ::: "memory"); }
// One chunk, issued by the lanes with copy != 0 (the group's leader): arrive expecting
// kChunkBytes, then the copy that completes them; lanes with arrive_only != 0 (the leader
// of a group without rows) only arrive.  Predicated, so the warp does not branch.
__device__ __forceinline__ void bulk_chunk(unsigned dst, const float4 *src, unsigned bar, unsigned copy,
                                           unsigned arrive_only) {
    asm volatile(
        "{\n .reg .pred pc, pa;\n setp.ne.u32 pc, %4, 0;\n setp.ne.u32 pa, %5, 0;\n"
        " @pc mbarrier.arrive.expect_tx.shared::cta.b64 _, [%2], %3;\n"
        " @pc cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %3, [%2];\n"
        " @pa mbarrier.arrive.shared::cta.b64 _, [%2];\n}\n" ::"r"(dst),
        "l"(__cvta_generic_to_global(src)), "r"(bar), "n"(kChunkBytes), "r"(copy), "r"(arrive_only)
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits for the phase of the given parity to complete; false after kWaitTries more tries
// (each try itself blocks for a bounded, hardware-chosen time).
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
    bool ok = mbar_try_wait(bar, parity);
    if (!ok) {
        for (int i = 0; i < kWaitTries && !ok; ++i) ok = mbar_try_wait(bar, parity);
    }
    return ok;
}
// 16-byte shared-memory accesses by 32-bit shared addresses (the chunk buffers and impulse
// words are reached through addresses the compiler cannot trace back to shared memory)
__device__ __forceinline__ float4 lds4(unsigned a) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ float lds1(unsigned a) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];\n" : "=f"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void sts4(unsigned a, float4 v) {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w) : "memory");
}

struct BodySm {
    float v[kMaxBodies][3], w[kMaxBodies][3];
    float invm[kMaxBodies];
    float Iinv[kMaxBodies][6];
    float com[kMaxBodies][3];
    // one lane updates an env's bodies: every body's velocity is written back
    __device__ __forceinline__ bool writes(int) const { return true; }
};

// The bodies of a pile env in the prep's shared memory (forces, then the rows' geometry and
// masses); the sweeps read and write the movable bodies' velocities in global memory.
struct PileBodies {
    float (*v)[3];
    float (*w)[3];
    float *invm;
    float (*Iinv)[6];
    float (*com)[3];
    const unsigned char *mov;   // 1: dynamic or fixed axis
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
static_assert(sizeof(Row) >= kRowF4 * sizeof(float4), "a fast row lives in a general row's storage");
static_assert(offsetof(Row, t1) == 3 * 4 && offsetof(Row, ra_n) == 9 * 4 && offsetof(Row, rb_n) == 18 * 4 &&
                  offsetof(Row, ia_n) == 27 * 4 && offsetof(Row, ib_n) == 36 * 4 && offsetof(Row, kn) == 45 * 4 &&
                  offsetof(Row, bias) == 48 * 4 && offsetof(Row, mu) == 49 * 4 && offsetof(Row, a) == 53 * 4 &&
                  offsetof(Row, b) == 54 * 4 && sizeof(Row) == kRowF4 * sizeof(float4),
              "gs_row reads Row fields by these word offsets");
__host__ __device__ inline int env_stride_f4(int lam_cap) { return ((lam_cap + kSlotF4 + 7) & ~7) + 1; }

__device__ __forceinline__ V3 smv(const float (*a)[3], int i) { return v3(a[i][0], a[i][1], a[i][2]); }
__device__ __forceinline__ void smv_set(float (*a)[3], int i, V3 x) { a[i][0] = x.x; a[i][1] = x.y; a[i][2] = x.z; }

// effective mass 1 / (m_a^-1 + m_b^-1 + (r_a x d) I_a^-1 (r_a x d) + (r_b x d) I_b^-1 (r_b x d))
__device__ __forceinline__ float eff_mass(float ima, float imb, V3 rad, V3 iad, V3 rbd, V3 ibd) {
    const float den = ima + imb + dot(rad, iad) + dot(rbd, ibd);
    return den > 0.0f ? 1.0f / den : 0.0f;
}

// word offsets of the Row fields (static_assert above)
enum RowWord : int {
    kWN = 0, kWT1 = 3, kWT2 = 6, kWRAN = 9, kWRAT1 = 12, kWRAT2 = 15, kWRBN = 18, kWRBT1 = 21, kWRBT2 = 24,
    kWIAN = 27, kWIAT1 = 30, kWIAT2 = 33, kWIBN = 36, kWIBT1 = 39, kWIBT2 = 42, kWKN = 45, kWKT1 = 46,
    kWKT2 = 47, kWBIAS = 48, kWMU = 49, kWLN = 50, kWA = 53, kWB = 54
};

// One contact's rows (Row), built in registers and written as 15 float4.
template <class BS>
__device__ __forceinline__ void build_row(Row &R, const DContact &c, const BS &B, int a, int b, float mu,
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
    float f[4 * kRowF4];
    auto put = [&](int o, V3 v) { f[o] = v.x; f[o + 1] = v.y; f[o + 2] = v.z; };
    put(kWN, n); put(kWT1, t1); put(kWT2, t2);
    put(kWRAN, ran); put(kWRAT1, rat1); put(kWRAT2, rat2);
    put(kWRBN, rbn); put(kWRBT1, rbt1); put(kWRBT2, rbt2);
    put(kWIAN, ian); put(kWIAT1, iat1); put(kWIAT2, iat2);
    put(kWIBN, ibn); put(kWIBT1, ibt1); put(kWIBT2, ibt2);
    const float ima = B.invm[a], imb = B.invm[b];
    f[kWKN] = eff_mass(ima, imb, ran, ian, rbn, ibn);
    f[kWKT1] = eff_mass(ima, imb, rat1, iat1, rbt1, ibt1);
    f[kWKT2] = eff_mass(ima, imb, rat2, iat2, rbt2, ibt2);
    f[kWBIAS] = (phi > 0.0f) ? phi / hs : baumgarte * phi / hs;
    f[kWMU] = mu;
    f[kWLN] = 0.0f; f[kWLN + 1] = 0.0f; f[kWLN + 2] = 0.0f;
    f[kWA] = __int_as_float(a); f[kWB] = __int_as_float(b);
#pragma unroll
    for (int k = kWB + 1; k < 4 * kRowF4; ++k) f[k] = 0.0f;
    float4 *q = reinterpret_cast<float4 *>(&R);
#pragma unroll
    for (int k = 0; k < kRowF4; ++k) q[k] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
}

// 1. of a substep for body bi (slot lb of the body store): gravity, applied force and
// torque and the gyroscopic term (dynamic bodies), the torque about the axis (fixed axis);
// writes its velocity, angular velocity, centre of mass (world), inverse mass and world
// inverse inertia (a fixed-axis body: a a^T / I_aa; others without rotation: zero).
template <class BS>
__device__ __forceinline__ void body_forces(const SimParams &p, int bi, int lb, float hs, BS &B) {
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

// 4. of a substep for body bi (constants P) from its velocity v, angular velocity w and
// centre of mass com: |omega| clamp (w is updated), semi-implicit Euler of the centre of
// mass and q <- normalize(q + hs/2 (omega, 0) q); writes the position and returns the new
// quaternion (a static body keeps its own); a non-finite result sets the status bit.
__device__ __forceinline__ float4 integrate_core(const SimParams &p, const BodyProps &P, int bi, float hs, V3 &w,
                                                 V3 v, V3 com_now) {
    float4 q = make_float4(p.quat[4 * bi], p.quat[4 * bi + 1], p.quat[4 * bi + 2], p.quat[4 * bi + 3]);
    if (P.type == FW_BODY_STATIC) return q;
    if ((P.type == FW_BODY_DYNAMIC || P.type == FW_BODY_FIXED_AXIS) && p.max_angvel > 0.0f) {
        const float wn = sqrtf(dot(w, w));
        if (wn > p.max_angvel) w = (p.max_angvel / wn) * w;
    }
    const V3 com = com_now + hs * v;
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
    const bool bad = !(isfinite(pos.x) && isfinite(pos.y) && isfinite(pos.z) && isfinite(q.x) && isfinite(q.y) &&
                       isfinite(q.z) && isfinite(q.w));
    if (bad) atomicOr(p.status, kStatusNonFinite);
    return q;
}

// integrate_core for body bi in slot lb of a body store
template <class BS>
__device__ __forceinline__ float4 body_integrate(const SimParams &p, int bi, int lb, float hs, BS &B) {
    const BodyProps P = p.props[bi];
    V3 w = smv(B.w, lb);
    const float4 q = integrate_core(p, P, bi, hs, w, smv(B.v, lb), smv(B.com, lb));
    if (P.type != FW_BODY_STATIC) smv_set(B.w, lb, w);
    return q;
}

// a row's 15 float4 as 60 words
__device__ __forceinline__ void load_row_words(const Row *R, float (&f)[4 * kRowF4]) {
    const float4 *q = reinterpret_cast<const float4 *>(R);
#pragma unroll
    for (int k = 0; k < kRowF4; ++k) {
        const float4 v = q[k];
        f[4 * k] = v.x; f[4 * k + 1] = v.y; f[4 * k + 2] = v.z; f[4 * k + 3] = v.w;
    }
}

// One contact's Gauss-Seidel update in the general form on the two bodies' velocities:
// the normal row, then the two friction rows projected jointly on the disk; L =
// (lambda_n, lambda_t1, lambda_t2, -).  The disk projection scales by
// min(1, mu lambda_n / |lambda_t|) through a reciprocal square root, as the fast form does.
// A row with a zero normal effective mass changes nothing.
__device__ __forceinline__ void gs_core(const float (&f)[4 * kRowF4], float4 &L, V3 &va, V3 &wa, V3 &vb, V3 &wb,
                                        float ima, float imb, bool use_bias) {
    auto w3 = [&](int o) { return v3(f[o], f[o + 1], f[o + 2]); };
    if (f[kWKN] == 0.0f) return;
    // normal row
    const V3 n = w3(kWN);
    float jv = dot(n, va - vb) + dot(w3(kWRAN), wa) - dot(w3(kWRBN), wb);
    if (use_bias) jv += f[kWBIAS];
    const float ln = fmaxf(L.x - f[kWKN] * jv, 0.0f);
    const float dl = ln - L.x;
    L.x = ln;
    va = va + (dl * ima) * n;
    wa = wa + dl * w3(kWIAN);
    vb = vb - (dl * imb) * n;
    wb = wb - dl * w3(kWIBN);
    // friction rows, projected jointly on the disk of radius mu lambda_n
    const V3 t1 = w3(kWT1), t2 = w3(kWT2);
    const V3 dv = va - vb;
    const float j1 = dot(t1, dv) + dot(w3(kWRAT1), wa) - dot(w3(kWRBT1), wb);
    const float j2 = dot(t2, dv) + dot(w3(kWRAT2), wa) - dot(w3(kWRBT2), wb);
    float l1 = L.y - f[kWKT1] * j1, l2 = L.z - f[kWKT2] * j2;
    const float sc = fminf(1.0f, (f[kWMU] * ln) * rsqrtf(__fmaf_rn(l1, l1, l2 * l2)));
    l1 *= sc;
    l2 *= sc;
    const float d1 = l1 - L.y, d2 = l2 - L.z;
    L.y = l1;
    L.z = l2;
    const V3 pt = d1 * t1 + d2 * t2;
    va = va + ima * pt;
    wa = wa + d1 * w3(kWIAT1) + d2 * w3(kWIAT2);
    vb = vb - imb * pt;
    wb = wb - (d1 * w3(kWIBT1) + d2 * w3(kWIBT2));
}

// gs_core on one row with the bodies' velocities in the body store (read, updated, written
// back where the store allows).
template <class BS>
__device__ __forceinline__ void gs_row(const Row &R, float4 &L, BS &B, bool use_bias) {
    float f[4 * kRowF4];
    load_row_words(&R, f);
    if (f[kWKN] == 0.0f) return;
    const int a = __float_as_int(f[kWA]), b = __float_as_int(f[kWB]);
    V3 va = smv(B.v, a), wa = smv(B.w, a), vb = smv(B.v, b), wb = smv(B.w, b);
    gs_core(f, L, va, wa, vb, wb, B.invm[a], B.invm[b], use_bias);
    if (B.writes(a)) { smv_set(B.v, a, va); smv_set(B.w, a, wa); }
    if (B.writes(b)) { smv_set(B.v, b, vb); smv_set(B.w, b, wb); }
}

// One Gauss-Seidel sweep over the env's rows in global memory, impulses in the rows (lane
// 0 only; the form for envs whose rows exceed the shared-memory impulse capacity).
__device__ void sweep(Row *rows, int nr, BodySm &B, bool use_bias) {
    for (int r = 0; r < nr; ++r) {
        Row &R = rows[r];
        float4 L = make_float4(R.ln, R.lt1, R.lt2, 0.0f);
        gs_row(R, L, B, use_bias);
        R.ln = L.x; R.lt1 = L.y; R.lt2 = L.z;
    }
}

// n_sweeps Gauss-Seidel sweeps in the general form (lane 0 only), the same updates as
// sweep(): the rows, read-only here, stream through the env's shared-memory ring with
// cp.async kRing - 1 steps ahead, so that no step waits on a global load; the impulses live
// in lam (one float4 per row, shared memory).
__device__ __noinline__ void sweep_general(const Row *rows, int nr, int n_sweeps, float4 *ring, float4 *lam,
                                           BodySm &B, bool use_bias) {
    const int total = nr * n_sweeps;
    if (total == 0) return;
    const float4 *src = reinterpret_cast<const float4 *>(rows);
    int pf = 0;   // row of the next step to prefetch
    for (int s = 0; s < kRing - 1; ++s) {
        if (s < total) {
            for (int k = 0; k < kRowF4; ++k) cp_async16(ring + s * kRowF4 + k, src + (size_t)pf * kRowF4 + k);
            if (++pf == nr) pf = 0;
        }
        cp_async_commit();
    }
    int r = 0;
    for (int s = 0; s < total; ++s) {
        const int sp = s + kRing - 1;   // its slot held step s - 1, already consumed
        if (sp < total) {
            float4 *dst = ring + (sp % kRing) * kRowF4;
            for (int k = 0; k < kRowF4; ++k) cp_async16(dst + k, src + (size_t)pf * kRowF4 + k);
            if (++pf == nr) pf = 0;
        }
        cp_async_commit();
        asm volatile("cp.async.wait_group %0;\n" ::"n"(kRing - 1) : "memory");
        const Row &R = *reinterpret_cast<const Row *>(ring + (s % kRing) * kRowF4);
        float4 L = lam[r];
        gs_row(R, L, B, use_bias);
        lam[r] = L;
        if (++r == nr) r = 0;
    }
    cp_async_wait_all();
}

// Fast row of one contact, from the side of the movable body m (a or b of the pair).
// For each row direction j in (n, 1, 2) = (d_n, d_1, d_2) = s (n, t1, t2), s = +1 when m
// is body a: the Jacobian J_j = (d_j, r x d_j) acting on m's velocity u = (v, w), the
// update vector W_j = M^-1 J_j^T = (ima d_j, I^-1 (r x d_j)) (an impulse lambda along j
// changes u by lambda W_j), the effective mass k_j = 1 / (J_j . W_j) and the partner's
// constant e_j = -d_j . (v_o + w_o x r_o).  Stored scaled by -k_j, so that a row's
// "scaled velocity" S_j = -k_j (J_j . u + e_j [+ bias for n]) gives the impulse change
// directly (lambda_n' = max(0, lambda_n + S_n)):
// directly (lambda_n' = max(0, lambda_n + S_n)).  Two halves of six float4, one per
// velocity part, then three of coefficients every lane needs:
//   linear half   f[0] = (-k_n d_n, -k_n (e_n + bias))   f[3] = (W_n linear, -k_n e_n)
//                 f[1] = (-k_1 d_1, -k_1 e_1)            f[4] = (W_1 linear, 0)
//                 f[2] = (-k_2 d_2, -k_2 e_2)            f[5] = (W_2 linear, 0)
//   angular half  f[6] = (-k_n (r x d_n), 0)             f[9]  = (W_n angular, 0)
//                 f[7] = (-k_1 (r x d_1), 0)             f[10] = (W_1 angular, 0)
//                 f[8] = (-k_2 (r x d_2), 0)             f[11] = (W_2 angular, 0)
//   f[12] = (K_1, K_2, mu, C_n0)  f[13] = (C_n1, C_n2, C_10, C_11)  f[14] = (C_12, C_20, C_21, C_22)
// so that a half's j-th Jacobian part is its float4 j and its update-vector part float4 3 + j,
// and its constant terms (zero in the angular half) sit in the .w words.
// K_k = -k_k J_k . W_n is the change of friction row k's scaled velocity per unit normal
// impulse of the same contact; C_jk = -k'_j J'_j . W_k (J'_j, k'_j of the NEXT row, r+1,
// wrapping from the last row to the first) the change of the next row's scaled velocity
// j per unit impulse along this row's direction k -- the entries of J M^-1 J^T between
// neighbouring rows.  They let the sweep carry the next row's three scaled velocities
// from one row to the next with two dependent FMAs, instead of rebuilding them from the
// updated body velocity.  A contact neither body can act on is an all-zero row.
__device__ __forceinline__ void build_fast_row(float4 *f, float4 &lam0, const DContact &c, const BodySm &B, int a,
                                               int b, int m, float mu, float hs, float baumgarte) {
    lam0 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k = 0; k < kRowF4; ++k) f[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (m != a && m != b) return;   // neither body of this pair can move
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
    const V3 d[3] = {sg * n, sg * t1, sg * t2};
    const V3 uo = smv(B.v, o) + cross(smv(B.w, o), ro);
    const float ima = B.invm[m];
    V3 a3[3], i3[3];
    float k[3], e[3];
    for (int j = 0; j < 3; ++j) {
        a3[j] = cross(rm, d[j]);
        i3[j] = sym_mul(B.Iinv[m], a3[j]);
        k[j] = eff_mass(ima, 0.0f, a3[j], i3[j], v3(0, 0, 0), v3(0, 0, 0));
        e[j] = -dot(d[j], uo);
    }
    if (k[0] == 0.0f) return;   // the movable body cannot respond along n
    const float bias = (phi > 0.0f) ? phi / hs : baumgarte * phi / hs;
    const V3 wnl = ima * d[0];
    // K_k = -k_k (ima d_k . d_n + (r x d_k) . I^-1 (r x d_n))
    const float K1 = -k[1] * (dot(d[1], wnl) + dot(a3[1], i3[0]));
    const float K2 = -k[2] * (dot(d[2], wnl) + dot(a3[2], i3[0]));
    const V3 jn = -k[0] * d[0], jan = -k[0] * a3[0];
    const V3 j1 = -k[1] * d[1], ja1 = -k[1] * a3[1];
    const V3 j2 = -k[2] * d[2], ja2 = -k[2] * a3[2];
    const V3 w1l = ima * d[1], w2l = ima * d[2];
    f[0] = make_float4(jn.x, jn.y, jn.z, -k[0] * (e[0] + bias));
    f[1] = make_float4(j1.x, j1.y, j1.z, -k[1] * e[1]);
    f[2] = make_float4(j2.x, j2.y, j2.z, -k[2] * e[2]);
    f[3] = make_float4(wnl.x, wnl.y, wnl.z, -k[0] * e[0]);
    f[4] = make_float4(w1l.x, w1l.y, w1l.z, 0.f);
    f[5] = make_float4(w2l.x, w2l.y, w2l.z, 0.f);
    f[6] = make_float4(jan.x, jan.y, jan.z, 0.f);
    f[7] = make_float4(ja1.x, ja1.y, ja1.z, 0.f);
    f[8] = make_float4(ja2.x, ja2.y, ja2.z, 0.f);
    f[9] = make_float4(i3[0].x, i3[0].y, i3[0].z, 0.f);
    f[10] = make_float4(i3[1].x, i3[1].y, i3[1].z, 0.f);
    f[11] = make_float4(i3[2].x, i3[2].y, i3[2].z, 0.f);
    f[12] = make_float4(K1, K2, mu, 0.f);
}

// C_jk of row r against its next row (see build_fast_row): scaled next-row Jacobian j
// dotted with this row's update vector k.
__device__ __forceinline__ void couple_fast_row(float4 *fr, const float4 *fn) {
    V3 J[3][2], W[3][2];
    for (int j = 0; j < 3; ++j) {
        J[j][0] = v3(fn[j].x, fn[j].y, fn[j].z);
        J[j][1] = v3(fn[kHalfF4 + j].x, fn[kHalfF4 + j].y, fn[kHalfF4 + j].z);
        W[j][0] = v3(fr[3 + j].x, fr[3 + j].y, fr[3 + j].z);
        W[j][1] = v3(fr[kHalfF4 + 3 + j].x, fr[kHalfF4 + 3 + j].y, fr[kHalfF4 + 3 + j].z);
    }
    float C[3][3];
    for (int j = 0; j < 3; ++j)
        for (int kk = 0; kk < 3; ++kk) C[j][kk] = dot(J[j][0], W[kk][0]) + dot(J[j][1], W[kk][1]);
    fr[12].w = C[0][0];
    fr[13] = make_float4(C[0][1], C[0][2], C[1][0], C[1][1]);
    fr[14] = make_float4(C[1][2], C[2][0], C[2][1], C[2][2]);
}

// ---- pile rows: the fast form for two movable bodies
// A pile pair's contact, kPileRowF4 float4.  Quarter q of the two bodies' velocities (q = 0
// linear and 1 angular velocity of body a, 2 and 3 those of body b; one lane of the sweep
// each) holds at float4 kPfQ q + k (k = 0, 1, 2: the normal n and the tangents t1, t2) the
// quarter's part of the scaled Jacobian -k_k J_k (.w: the normal row's bias term
// -k_n b in quarter 0, zero elsewhere) and at kPfQ q + 3 + k the update vector
// (M^-1 J_k^T)_q, where for direction d = d_k
//   q = 0: J = d,          M^-1 J^T = m_a^-1 d         q = 1: J = r_a x d,     I_a^-1 (r_a x d)
//   q = 2: J = -d,         M^-1 J^T = -m_b^-1 d        q = 3: J = -(r_b x d), -I_b^-1 (r_b x d)
// (the update of gs_core, whose impulse is -k_k (J_k v + bias)).  Float4 kPfC .. kPfC + 2
// hold K_1, K_2, mu and the couplings C_jk to the pair's next row in the order of the fast
// rows' float4 12 .. 14; float4 kPfL the impulses (lambda_n, lambda_t1, lambda_t2, 0),
// which the sweeps update.  A contact with a zero normal effective mass is an all-zero row.
constexpr int kPfQ = 6, kPfC = 24, kPfL = 27;
static_assert(kPfL + 1 == kPileRowF4, "pile row layout");

// Bodies a and b: centres of mass (world) ca, cb, world inverse inertias Ia, Ib (six stored
// words), inverse masses ima, imb.
__device__ __forceinline__ void build_pile_row(float4 *f, const DContact &c, V3 ca, V3 cb, const float *Ia,
                                               const float *Ib, float ima, float imb, float mu, float hs,
                                               float baumgarte) {
    const V3 n = ld3(c.n), xa = ld3(c.xa);
    const float phi = c.phi;
    const V3 xb = xa - phi * n;
    const V3 ra = xa - ca, rb = xb - cb;
    V3 t1, t2;
    tangent_basis(n, t1, t2);
    const V3 d[3] = {n, t1, t2};
    V3 J[3][4], W[3][4];
    float k[3];
    for (int j = 0; j < 3; ++j) {
        const V3 rad = cross(ra, d[j]), rbd = cross(rb, d[j]);
        const V3 iad = sym_mul(Ia, rad), ibd = sym_mul(Ib, rbd);
        k[j] = eff_mass(ima, imb, rad, iad, rbd, ibd);
        J[j][0] = d[j]; J[j][1] = rad; J[j][2] = -1.0f * d[j]; J[j][3] = -1.0f * rbd;
        W[j][0] = ima * d[j]; W[j][1] = iad; W[j][2] = -imb * d[j]; W[j][3] = -1.0f * ibd;
    }
    for (int i = 0; i < kPileRowF4; ++i) f[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (k[0] == 0.0f) return;   // neither body can respond along n
    const float bias = (phi > 0.0f) ? phi / hs : baumgarte * phi / hs;
    float K[3] = {0.f, 0.f, 0.f};
    for (int q = 0; q < 4; ++q)
        for (int j = 0; j < 3; ++j) {
            const V3 sj = -k[j] * J[j][q];
            f[kPfQ * q + j] = make_float4(sj.x, sj.y, sj.z, (q == 0 && j == 0) ? -k[0] * bias : 0.0f);
            f[kPfQ * q + 3 + j] = make_float4(W[j][q].x, W[j][q].y, W[j][q].z, 0.0f);
            K[j] += dot(sj, W[0][q]);   // K_j = -k_j J_j . M^-1 J_n^T
        }
    f[kPfC] = make_float4(K[1], K[2], mu, 0.0f);
}

// C_jk of pile row r against the pair's next row fn (nullptr: r is the pair's last row and
// keeps zero couplings): next row's scaled Jacobian j dotted with this row's update vector k.
__device__ __forceinline__ void couple_pile_row(float4 *fr, const float4 *fn) {
    float C[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    if (fn)
        for (int q = 0; q < 4; ++q)
            for (int j = 0; j < 3; ++j)
                for (int kk = 0; kk < 3; ++kk) {
                    const float4 a = fn[kPfQ * q + j], b = fr[kPfQ * q + 3 + kk];
                    C[j][kk] += a.x * b.x + a.y * b.y + a.z * b.z;
                }
    fr[kPfC].w = C[0][0];
    fr[kPfC + 1] = make_float4(C[0][1], C[0][2], C[1][0], C[1][1]);
    fr[kPfC + 2] = make_float4(C[1][2], C[2][0], C[2][1], C[2][2]);
}

// smallest v over the warp's groups (lanes of a group hold the same v)
template <int G>
__device__ __forceinline__ int warp_min(int v) {
#pragma unroll
    for (int off = G; off < 32; off <<= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}

// A row as one lane holds it, in the pieces a step uses at different times: the scaled
// Jacobian of the lane's half (J, float4 0-2 of the half), whose scaled velocities at the
// body velocity are formed the step BEFORE the row is solved, and the half's update vectors
// (W, float4 3-5 of the half) with the coefficients every lane needs (C, float4 12-14), used
// when it is solved.  nc is the normal row's constant without the bias (float4 3 .w of the
// half), for the bias-free sweeps.
struct RowJ {
    float4 j[3];
    float nc;
};
struct RowCW {
    float4 c[3];
    float4 w[3];
};

__device__ __forceinline__ void read_j(unsigned hp, RowJ &r, bool need_nc) {
#pragma unroll
    for (int k = 0; k < 3; ++k) r.j[k] = lds4(hp + 16u * k);
    if (need_nc) r.nc = lds1(hp + 16u * 3 + 12u);
}
__device__ __forceinline__ void read_cw(unsigned hp, unsigned cp, RowCW &r) {
#pragma unroll
    for (int k = 0; k < 3; ++k) r.w[k] = lds4(hp + 16u * (3 + k));
#pragma unroll
    for (int k = 0; k < 3; ++k) r.c[k] = lds4(cp + 16u * k);
}

// scaled velocities of a row at the body velocity (u and its partner lane's half), without
// couplings: each lane dots its half, the pair adds the two parts (the same sum on both)
template <bool kBias>
__device__ __forceinline__ void row_base(const RowJ &g, V3 u, float &bn, float &b1, float &b2) {
    const float pn = __fmaf_rn(g.j[0].z, u.z, __fmaf_rn(g.j[0].y, u.y, __fmaf_rn(g.j[0].x, u.x, kBias ? g.j[0].w : g.nc)));
    const float p1 = __fmaf_rn(g.j[1].z, u.z, __fmaf_rn(g.j[1].y, u.y, __fmaf_rn(g.j[1].x, u.x, g.j[1].w)));
    const float p2 = __fmaf_rn(g.j[2].z, u.z, __fmaf_rn(g.j[2].y, u.y, __fmaf_rn(g.j[2].x, u.x, g.j[2].w)));
    bn = pn + __shfl_xor_sync(0xffffffffu, pn, 1);
    b1 = p1 + __shfl_xor_sync(0xffffffffu, p1, 1);
    b2 = p2 + __shfl_xor_sync(0xffffffffu, p2, 1);
}

// The chunked row stream of one env (one lane group).  The env's rows, read cyclically
// (sweep after sweep), are cut into chunks of kChunk consecutive stream positions; chunk k
// of the kernel's sequence goes to buffer k mod kChunkBufs and completes phase
// k / kChunkBufs of that buffer's mbarrier.  Lane 0 of the group issues the copies (one
// cp.async.bulk of kChunkBytes each, contiguous thanks to the kRowPad repeated rows after
// the env's region);
// a group without rows only arrives, so its phases complete at once and its buffers keep
// the zeros they were given.
struct RowStream {
    const float4 *rows;   // the env's rows (global), followed by kRowPad repeated ones
    float4 *buf;          // kChunkBufs chunk buffers (shared)
    unsigned bar;         // shared address of the first of their kChunkBufs mbarriers
    int nr;               // rows of the env (0: none)
    int pf;               // row at which the next chunk to issue starts
    int seq;              // chunks issued so far in this kernel (the next one's number)
    int ib;               // buffer of the next chunk to issue (seq mod kChunkBufs)
    bool leader;          // lane 0 of the group
    bool on;              // issuing (cleared after a wait gave up)
    int seq_on;           // chunks issued while on (only those complete their phases)
};

__device__ __forceinline__ void issue_chunk(RowStream &rs) {
    const unsigned bar = rs.bar + 8u * rs.ib;
    bulk_chunk(smem_addr(rs.buf) + 16u * kChunkF4 * rs.ib, rs.rows + (size_t)kRowF4 * rs.pf, bar,
               rs.leader && rs.on && rs.nr > 0, rs.leader && rs.on && rs.nr == 0);
    if (rs.nr >= kChunk) {
        rs.pf += kChunk;
        rs.pf = rs.pf >= rs.nr ? rs.pf - rs.nr : rs.pf;
    } else if (rs.nr > 0) {
        rs.pf = (rs.pf + kChunk) % rs.nr;
    }
    if (rs.on) rs.seq_on = rs.seq + 1;
    ++rs.seq;
    rs.ib = rs.ib + 1 == kChunkBufs ? 0 : rs.ib + 1;
}

struct SweepRegs {
    V3 u;                 // the lane's half of the body velocity before the current row
    float sn, s1, s2;     // current row's scaled velocities at that velocity, incl. couplings
};

// One Gauss-Seidel step of a group, software-pipelined over three rows.  Row j (C and W in
// f, impulse word Lf) is solved from its carried scaled velocities; meanwhile the next row's
// scaled velocities are formed at the body velocity before row j from its Jacobian half jn
// (read a step earlier), and the loads for later steps are issued: row j + 1's C and W
// (into fn, at shared addresses hn / cn), row j + 2's Jacobian half (into jnn, at hnn) and
// row j + 1's impulse word (Lg).  Only S -> impulse changes -> next row's S (through the
// couplings C) is serial; no load result is needed within the step it is issued in.  kFast:
// every group of the warp takes this step for real; otherwise a step past a group's total is
// computed and discarded (act = false), and with a single row the next row is the current
// one.  The leader lane stores the new impulse word at lam_cur.
template <bool kBias, bool kFast>
__device__ __forceinline__ void gs_step(const RowCW &f, const float4 &Lf, const RowJ &jn, RowCW &fn, RowJ &jnn,
                                        float4 &Lg, SweepRegs &st, unsigned hn, unsigned cn, unsigned hnn,
                                        unsigned lam_next, unsigned lam_cur, bool leader, bool act, bool single) {
    // the next row's scaled velocities at the body velocity before this row: independent of
    // this row's solve, so they are formed first and overlap its dependency chain
    float bn, b1, b2;
    row_base<kBias>(jn, st.u, bn, b1, b2);
    read_cw(hn, cn, fn);
    read_j(hnn, jnn, !kBias);
    Lg = lds4(lam_next);
    // the current row, from its carried scaled velocities
    const float4 L = Lf;
    const float dl = fmaxf(st.sn, -L.x);                  // lambda_n' - lambda_n
    const float da = (kFast || act) ? dl : 0.0f;
    const V3 u = st.u;
    const V3 ud = v3(__fmaf_rn(da, f.w[0].x, u.x), __fmaf_rn(da, f.w[0].y, u.y), __fmaf_rn(da, f.w[0].z, u.z));
    const float xn = __fmaf_rn(f.c[0].w, dl, bn), x1 = __fmaf_rn(f.c[1].z, dl, b1), x2 = __fmaf_rn(f.c[2].y, dl, b2);
    const float ln = L.x + dl;
    const float t1 = __fmaf_rn(f.c[0].x, dl, st.s1 + L.y);
    const float t2 = __fmaf_rn(f.c[0].y, dl, st.s2 + L.z);
    const float sc = fminf(1.0f, (f.c[0].z * ln) * rsqrtf(__fmaf_rn(t1, t1, t2 * t2)));
    const float e1 = __fmaf_rn(t1, sc, -L.y), e2 = __fmaf_rn(t2, sc, -L.z);
    // the next row's scaled velocities: plus the couplings
    st.sn = __fmaf_rn(f.c[1].y, e2, __fmaf_rn(f.c[1].x, e1, xn));
    st.s1 = __fmaf_rn(f.c[2].x, e2, __fmaf_rn(f.c[1].w, e1, x1));
    st.s2 = __fmaf_rn(f.c[2].w, e2, __fmaf_rn(f.c[2].z, e1, x2));
    // the lane's half of the body velocity after this row
    const float e1a = (kFast || act) ? e1 : 0.0f, e2a = (kFast || act) ? e2 : 0.0f;
    st.u = v3(__fmaf_rn(e2a, f.w[2].x, __fmaf_rn(e1a, f.w[1].x, ud.x)),
              __fmaf_rn(e2a, f.w[2].y, __fmaf_rn(e1a, f.w[1].y, ud.y)),
              __fmaf_rn(e2a, f.w[2].z, __fmaf_rn(e1a, f.w[1].z, ud.z)));
    const float4 nl = make_float4(ln, L.y + e1, L.z + e2, 0.0f);
    if (leader && (kFast || act)) sts4(lam_cur, nl);
    if (!kFast && single) Lg = nl;
}

// `passes` Gauss-Seidel sweeps over nr fast rows by one group of G lanes (one env), one
// row per step, total = nr * passes steps.  All lanes of the warp run the same number of
// steps, `trips` rounded up to whole chunks (rows past a group's own total are computed
// and discarded), so every shuffle and warp vote is reached by the whole warp.  The even
// lanes of a group keep the body's linear velocity, the odd lanes its angular velocity;
// scaled velocities and impulses are identical on all of them.  Chunk c of the call is read
// while chunk c + 1 is in flight (issued into chunk c - 1's buffer as chunk c starts); its
// step kChunk - 2 waits for chunk c + 1, whose first row's Jacobian is loaded there (two
// rows ahead).  The chunks that every group of the warp takes for real (all kChunk steps
// below its total, at least kChunk + 2 rows) come first and run the kFast steps in a loop
// of their own: shared-memory offsets constant but for the one impulse-index wrap a chunk
// may hold (two base addresses), one __syncwarp per chunk ordering the leader's impulse
// stores before other lanes' later reads (a row's impulse word is read again at least
// kChunk + 1 steps after its store).  The remaining chunks (the last of the sweeps when the
// warp's envs have different totals, envs of fewer rows) take the general steps (index
// wrap, masking, a __syncwarp per step) in a second loop; with the general steps in the
// same loop as the fast ones, the fast chunks ran about 4% slower.  Returns false if a wait
// for a chunk gave up (bounded); the chunks still in flight are then waited for (bounded
// again) before returning.
template <int G, bool kBias>
__device__ bool sweep_fast(RowStream &rs, int total, int trips, float4 *lam, V3 &va, V3 &wa, int gl) {
    if (trips == 0) return true;   // warp-uniform
    const int nr = rs.nr;
    const bool odd = gl & 1, leader = rs.leader;
    const int nch = (trips + kChunk - 1) / kChunk;   // chunks of steps; chunk nch is read ahead
    const int seq0 = rs.seq;
    // A group without rows runs steps whose results must leave its velocity as it is: zero
    // rows and zero impulses are a fixed point of the step (every update vector zero, the
    // impulses stay zero), but shared memory may hold any bits, NaN patterns included, and a
    // chunk whose other groups all run real steps runs this group's steps unmasked.  So its
    // chunk words and the impulse words its steps read (0 .. kChunk; past lam_cap they lie in
    // the chunk buffers) are made zeros.
    if (nr == 0) {
        for (int k = gl; k < kChunkBufs * kChunkF4; k += G) rs.buf[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int k = gl; k <= kChunk; k += G) lam[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncwarp();
    for (int k = 0; k < kChunkBufs && k <= nch; ++k) issue_chunk(rs);
    SweepRegs st;
    st.u = odd ? wa : va;
    // buffer and phase parity of the chunk being read (rb, rpar) and of the next one
    int rb = seq0 % kChunkBufs;
    unsigned rpar = (unsigned)((seq0 / kChunkBufs) & 1);
    bool ok = mbar_wait(rs.bar + 8u * rb, rpar);
    int done = seq0 + (ok ? 1 : 0);   // chunks waited for, in sequence
    const unsigned buf0 = smem_addr(rs.buf), lam0 = smem_addr(lam);
    constexpr unsigned kRowB = 16u * kRowF4, kChunkB = 16u * kChunkF4, kCoefB = 16u * 2 * kHalfF4;
    const unsigned hob = 16u * (odd ? kHalfF4 : 0);
    unsigned cur = buf0 + kChunkB * rb;
    // prologue: row 0 (C, W, impulse, its scaled velocities) and row 1's Jacobian half
    RowCW A, B;
    RowJ JA, JB;
    float4 LA, LB;
    read_cw(cur + hob, cur + kCoefB, A);
    read_j(cur + hob, JA, !kBias);
    LA = lds4(lam0);
    row_base<kBias>(JA, st.u, st.sn, st.s1, st.s2);
    read_j(cur + kRowB + hob, JB, !kBias);
    const bool single = nr == 1;
    int r = 0;    // row of the chunk's first step
    // Chunks 0 .. nfast - 1 are taken for real by every group of the warp (steps below each
    // group's total; a group with at least kChunk + 2 rows wraps its impulse index at most
    // once in a chunk's kChunk + 1 rows): they run the unmasked steps in a loop of their
    // own.  The rest (the sweeps' last partial chunk, envs of fewer rows) take the general
    // steps.
    int nfast = nr == 0 ? nch : (nr >= kChunk + 2 ? total / kChunk : 0);
    nfast = (int)__reduce_min_sync(0xffffffffu, (unsigned)nfast);
    int c = 0;
    for (; c < nfast; ++c) {
        if (c >= 1 && c + kChunkBufs - 1 <= nch) issue_chunk(rs);   // into chunk c - 1's buffer
        const int nb = rb + 1 == kChunkBufs ? 0 : rb + 1;
        const unsigned npar = nb == 0 ? rpar ^ 1u : rpar;
        cur = buf0 + kChunkB * rb;
        const unsigned nxt = buf0 + kChunkB * nb, nbar = rs.bar + 8u * nb;
        __syncwarp();
        // impulse word of step j: row r + j, or row r + j - nr from step wr = nr - r on
        const unsigned lpa = lam0 + 16u * r, lpb = lpa - 16u * nr;
        const int wr = nr - r;
        unsigned lcur = lpa;
#pragma unroll
        for (int j = 0; j < kChunk; j += 2) {
            // step kChunk - 2 loads row kChunk, the next chunk's first: wait for it (after a
            // wait gave up, no more waits: the results are discarded)
            if (j + 2 == kChunk && ok) {
                ok = mbar_wait(nbar, npar);
                done += ok ? 1 : 0;
            }
            const unsigned r1 = (j + 1 < kChunk) ? cur + kRowB * (j + 1) : nxt + kRowB * (j + 1 - kChunk);
            const unsigned r2 = (j + 2 < kChunk) ? cur + kRowB * (j + 2) : nxt + kRowB * (j + 2 - kChunk);
            const unsigned r3 = (j + 3 < kChunk) ? cur + kRowB * (j + 3) : nxt + kRowB * (j + 3 - kChunk);
            const unsigned l1 = (j + 1 < wr ? lpa : lpb) + 16u * (j + 1);
            gs_step<kBias, true>(A, LA, JB, B, JA, LB, st, r1 + hob, r1 + kCoefB, r2 + hob, l1, lcur, leader, true,
                                 false);
            const unsigned l2 = (j + 2 < wr ? lpa : lpb) + 16u * (j + 2);
            gs_step<kBias, true>(B, LB, JA, A, JB, LA, st, r2 + hob, r2 + kCoefB, r3 + hob, l2, l1, leader, true,
                                 false);
            lcur = l2;
        }
        if (nr > 0) {
            r += kChunk;
            r = r >= nr ? r - nr : r;
        }
        rb = nb;
        rpar = npar;
        rs.on = rs.on && ok;
    }
    for (; c < nch; ++c) {
        if (c >= 1 && c + kChunkBufs - 1 <= nch) issue_chunk(rs);
        const int nb = rb + 1 == kChunkBufs ? 0 : rb + 1;
        const unsigned npar = nb == 0 ? rpar ^ 1u : rpar;
        cur = buf0 + kChunkB * rb;
        const unsigned nxt = buf0 + kChunkB * nb, nbar = rs.bar + 8u * nb;
        const int q0 = c * kChunk;
#pragma unroll
        for (int j = 0; j < kChunk; j += 2) {
            if (j + 2 == kChunk && ok) {
                ok = mbar_wait(nbar, npar);
                done += ok ? 1 : 0;
            }
            const unsigned r1 = (j + 1 < kChunk) ? cur + kRowB * (j + 1) : nxt + kRowB * (j + 1 - kChunk);
            const unsigned r2 = (j + 2 < kChunk) ? cur + kRowB * (j + 2) : nxt + kRowB * (j + 2 - kChunk);
            const unsigned r3 = (j + 3 < kChunk) ? cur + kRowB * (j + 3) : nxt + kRowB * (j + 3 - kChunk);
            __syncwarp();
            int rn = r + 1 >= nr ? 0 : r + 1;
            gs_step<kBias, false>(A, LA, JB, B, JA, LB, st, r1 + hob, r1 + kCoefB, r2 + hob, lam0 + 16u * rn,
                                  lam0 + 16u * r, leader, q0 + j < total, single);
            r = rn;
            rn = r + 1 >= nr ? 0 : r + 1;
            __syncwarp();
            gs_step<kBias, false>(B, LB, JA, A, JB, LA, st, r2 + hob, r2 + kCoefB, r3 + hob, lam0 + 16u * rn,
                                  lam0 + 16u * r, leader, q0 + j + 1 < total, single);
            r = rn;
        }
        rb = nb;
        rpar = npar;
        rs.on = rs.on && ok;
    }
    const V3 other = v3(__shfl_xor_sync(0xffffffffu, st.u.x, 1), __shfl_xor_sync(0xffffffffu, st.u.y, 1),
                        __shfl_xor_sync(0xffffffffu, st.u.z, 1));
    va = odd ? other : st.u;
    wa = odd ? st.u : other;
    // normally every issued chunk has been waited for; after a wait gave up, wait (bounded)
    // for the copies issued after it, so that none lands after the kernel has moved on
    const bool all_ok = __all_sync(0xffffffffu, ok);
    for (int k = done; k < rs.seq_on; ++k) mbar_wait(rs.bar + 8u * (k % kChunkBufs), (unsigned)((k / kChunkBufs) & 1));
    __syncwarp();
    return all_ok;
}

template <int G>
__device__ __forceinline__ int warp_max(int v) {
#pragma unroll
    for (int off = G; off < 32; off <<= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}

// One substep's solve for kGroups envs per warp (G = 32 / kGroups lanes each) and
// blockDim.x / 32 warps per block.  No block-wide barrier: every warp is independent.
// n_sweeps weighted Jacobi sweeps (solver = 1) over an env's nr fast rows by its group of
// G lanes.  Every lane holds the whole body velocity u = (v, w).  Per sweep each lane takes
// rows gl, gl + G, ...: the contact's block update from the sweep-start velocity -- S_n from
// the scaled Jacobian, the normal clamp, S_1 and S_2 with the contact's own normal change
// (K_1, K_2), the projection on the disk -- and sums its velocity changes; the group adds
// the lanes' sums, and all impulses and the velocity move by omega = 1 / (rows that can
// act, those with a nonzero normal Jacobian).  The impulses live in the row's float4 13
// (a Jacobi row has no neighbour couplings), so no shared memory is needed.
template <int G, bool kBias>
__device__ void sweep_jacobi(float4 *rows_, int nr, int n_sweeps, V3 &va, V3 &wa, int gl) {
    // the sweep reads a row's coefficients (float4 0-12) and reads and writes its impulses
    // (float4 13) through separate pointers, so the next rows' loads may move ahead of the
    // impulse stores
    const float4 *__restrict__ rows = rows_;
    float4 *__restrict__ imp = rows_ + 13;
    int na = 0;
    for (int r = gl; r < nr; r += G) {
        const float4 f0 = rows[kRowF4 * r];
        na += (f0.x != 0.0f || f0.y != 0.0f || f0.z != 0.0f);
    }
#pragma unroll
    for (int off = 1; off < G; off <<= 1) na += __shfl_xor_sync(0xffffffffu, na, off);
    const float om = na > 0 ? 1.0f / (float)na : 0.0f;
    for (int it = 0; it < n_sweeps; ++it) {
        V3 dv = v3(0.0f, 0.0f, 0.0f), dw = v3(0.0f, 0.0f, 0.0f);
#pragma unroll 2
        for (int r = gl; r < nr; r += G) {
            const float4 *f = rows + kRowF4 * r;
            const float4 f0 = f[0], f1 = f[1], f2 = f[2], f3 = f[3], f4 = f[4], f5 = f[5];
            const float4 f6 = f[6], f7 = f[7], f8 = f[8], f9 = f[9], f10 = f[10], f11 = f[11];
            const float4 f12 = f[12], L = imp[kRowF4 * r];
            const float sn = dot(v3(f0.x, f0.y, f0.z), va) + (kBias ? f0.w : f3.w) + dot(v3(f6.x, f6.y, f6.z), wa);
            const float ln = fmaxf(L.x + sn, 0.0f);
            const float dn = ln - L.x;
            const float s1 = dot(v3(f1.x, f1.y, f1.z), va) + f1.w + dot(v3(f7.x, f7.y, f7.z), wa) + f12.x * dn;
            const float s2 = dot(v3(f2.x, f2.y, f2.z), va) + f2.w + dot(v3(f8.x, f8.y, f8.z), wa) + f12.y * dn;
            float l1 = L.y + s1, l2 = L.z + s2;
            const float sc = fminf(1.0f, (f12.z * ln) * rsqrtf(__fmaf_rn(l1, l1, l2 * l2)));   // disk
            l1 *= sc;
            l2 *= sc;
            const float d1 = l1 - L.y, d2 = l2 - L.z;
            dv = dv + dn * v3(f3.x, f3.y, f3.z) + d1 * v3(f4.x, f4.y, f4.z) + d2 * v3(f5.x, f5.y, f5.z);
            dw = dw + dn * v3(f9.x, f9.y, f9.z) + d1 * v3(f10.x, f10.y, f10.z) + d2 * v3(f11.x, f11.y, f11.z);
            imp[kRowF4 * r] = make_float4(L.x + om * dn, L.y + om * d1, L.z + om * d2, 0.0f);
        }
#pragma unroll
        for (int off = 1; off < G; off <<= 1) {
            dv.x += __shfl_xor_sync(0xffffffffu, dv.x, off);
            dv.y += __shfl_xor_sync(0xffffffffu, dv.y, off);
            dv.z += __shfl_xor_sync(0xffffffffu, dv.z, off);
            dw.x += __shfl_xor_sync(0xffffffffu, dw.x, off);
            dw.y += __shfl_xor_sync(0xffffffffu, dw.y, off);
            dw.z += __shfl_xor_sync(0xffffffffu, dw.z, off);
        }
        va = va + om * dv;
        wa = wa + om * dw;
    }
}

// Solve variants: Gauss-Seidel for worlds whose envs have at most one movable body, the
// same with the general form for several movable bodies (sweep_general: impulses in
// shared memory), and the weighted Jacobi solver; each is compiled only into its own
// kernel so the others keep their code and registers.
enum : int { kVarGS = 0, kVarMulti = 1, kVarJacobi = 2 };

// Rows per shared-memory chunk when an env of several movable bodies runs the two-body fast
// rows: two chunks fit the env slot's chunk buffers.
constexpr int kEnvPfChunk = 8;
static_assert(2 * kEnvPfChunk * kPileRowF4 <= kChunkBufs * kChunkF4, "two-body row chunks fit the env slot");
template <bool kBias>
__device__ void sweep_env_pf(const SimParams &p, const EnvDev &E, const int *row_base, float4 *frows, BodySm &B,
                             float4 *buf, int lane, int n_sweeps);

template <int kGroups, int kVar>
__global__ void __launch_bounds__(kSolveMaxWarps * 32, 1) solve_kernel(SimParams p) {
    constexpr bool kMulti = kVar == kVarMulti, kJacobi = kVar == kVarJacobi;
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
    // the group's chunk buffers and their mbarriers, behind its impulse words
    float4 *chunk_buf = env_base + p.lam_cap;
    const unsigned chunk_bar = smem_addr(chunk_buf + kChunkBufs * kChunkF4);
    if (!kJacobi && gl == 0) {
        for (int b = 0; b < kChunkBufs; ++b) mbar_init(chunk_bar + 8u * b);
        mbar_init_fence();
    }
    __shared__ EnvSm S_all[kSolveMaxWarps * kGroups];
    EnvSm &S = S_all[slot];
    BodySm &B = S.B;
    const float hs = p.hs;
    // 1. external forces; world inertia at the substep's start
    for (int lb = gl; lb < E.n_bodies; lb += G) body_forces(p, E.first_body + lb, lb, hs, B);
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
    float4 *ring = chunk_buf;   // the general form's cp.async ring (it has no chunk stream)
    const int m = E.movable;
    const bool fast = (m != -2) && (kJacobi || nr <= p.lam_cap);
    // several movable bodies with the warp to itself: the two-body fast rows (pile rows), swept
    // pair by pair with the pair's velocities carried by four lanes (sweep_env_pf); with
    // several envs per warp, general rows, impulses in shared memory when they fit
    const bool pf = kMulti && kGroups == 1 && valid && m == -2;
    const bool general_sm = kMulti && (m == -2) && nr <= p.lam_cap;
    float4 *frows = reinterpret_cast<float4 *>(rows);
    // 2. constraint preparation, one contact per lane, then the couplings between neighbours
    for (int k = 0; k < E.n_pairs; ++k) {
        const int pi = E.first_pair + k;
        const PairDev P = p.pairs[pi];
        const int cnt = S.row_base[k + 1] - S.row_base[k];
        for (int i = gl; i < cnt; i += G) {
            const DContact &c = p.contacts[(long long)pi * p.cap_pair + i];
            if (pf) {
                const int a = P.local_a, b = P.local_b;
                build_pile_row(frows + kPileRowF4 * (S.row_base[k] + i), c, smv(B.com, a), smv(B.com, b), B.Iinv[a],
                               B.Iinv[b], B.invm[a], B.invm[b], P.mu, hs, p.baumgarte);
            } else if (fast) {
                // Jacobi keeps its impulses in the row (float4 13, zeroed here) and has no
                // shared-memory impulse words: its lam region is empty (lam_cap = 0)
                float4 unused;
                if (m >= 0)
                    build_fast_row(frows + kRowF4 * (S.row_base[k] + i), kJacobi ? unused : lam[S.row_base[k] + i], c,
                                   B, P.local_a, P.local_b, m, P.mu, hs, p.baumgarte);
            } else {
                build_row(rows[S.row_base[k] + i], c, B, P.local_a, P.local_b, P.mu, hs, p.baumgarte);
                if (kMulti && general_sm) lam[S.row_base[k] + i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
        }
    }
    __threadfence_block();
    __syncwarp();
    if (pf) {   // couplings between a pair's neighbouring rows; the rows are read next by cp.async (L2)
        for (int k = 0; k < E.n_pairs; ++k) {
            const int r0 = S.row_base[k], cnt = S.row_base[k + 1] - r0;
            for (int i = gl; i < cnt; i += G)
                couple_pile_row(frows + kPileRowF4 * (r0 + i), i + 1 < cnt ? frows + kPileRowF4 * (r0 + i + 1) : nullptr);
        }
        __threadfence();
    }
    const bool streamed = !kJacobi && fast && m >= 0 && nr > 0;   // rows read through the chunk stream
    if (streamed) {
        for (int r = gl; r < nr; r += G) couple_fast_row(frows + kRowF4 * r, frows + kRowF4 * (r + 1 < nr ? r + 1 : 0));
    }
    __syncwarp();
    if (streamed) {   // the kRowPad rows after the env's rows repeat rows 0, 1, ... (mod nr)
        for (int k = gl; k < kRowPad * kRowF4; k += G) {
            const int j = k / kRowF4, f4 = k - j * kRowF4;
            frows[kRowF4 * (nr + j) + f4] = frows[kRowF4 * (j % nr) + f4];
        }
        // the rows are read next by bulk copies (async proxy) that lane 0 issues: make this
        // lane's row writes visible at device scope, then to the async proxy
        __threadfence();
        fence_async_global();
    }
    __threadfence_block();
    __syncwarp();
    // 3. Gauss-Seidel sweeps (no movable body: nothing to solve)
    const bool run_fast = valid && fast && m >= 0;
    RowStream rs;
    rs.rows = frows;
    rs.buf = chunk_buf;
    rs.bar = chunk_bar;
    rs.nr = run_fast ? nr : 0;
    rs.pf = 0;
    rs.seq = 0;
    rs.seq_on = 0;
    rs.ib = 0;
    rs.leader = gl == 0;
    rs.on = p.stall != 2;   // test hook: no chunk is issued, so its wait runs out
    bool waits_ok = true;
    {
        const int total = run_fast ? nr * p.n_iters : 0;
        const int trips = warp_max<G>(total);
        V3 va = v3(0, 0, 0), wa = v3(0, 0, 0);
        if (run_fast) { va = smv(B.v, m); wa = smv(B.w, m); }
        if (kJacobi) sweep_jacobi<G, true>(frows, run_fast ? nr : 0, p.n_iters, va, wa, gl);
        else waits_ok = sweep_fast<G, true>(rs, total, trips, lam, va, wa, gl);
        if (run_fast && gl == 0) { smv_set(B.v, m, va); smv_set(B.w, m, wa); }
    }
    if (pf) sweep_env_pf<true>(p, E, S.row_base, frows, B, chunk_buf, lane, p.n_iters);
    else if (valid && !fast && gl == 0) {
        if (kMulti && general_sm) sweep_general(rows, nr, p.n_iters, ring, lam, B, true);
        else for (int it = 0; it < p.n_iters; ++it) sweep(rows, nr, B, true);
    }
    __syncwarp();
    // 4. integration
    for (int lb = gl; lb < E.n_bodies; lb += G) {
        const float4 q = body_integrate(p, E.first_body + lb, lb, hs, B);
        S.q_new[lb][0] = q.x; S.q_new[lb][1] = q.y; S.q_new[lb][2] = q.z; S.q_new[lb][3] = q.w;
    }
    __syncwarp();
    // 5. optional bias-free sweeps
    if (p.n_vel_iters > 0) {
        const int total = run_fast ? nr * p.n_vel_iters : 0;
        const int trips = warp_max<G>(total);
        V3 va = v3(0, 0, 0), wa = v3(0, 0, 0);
        if (run_fast) { va = smv(B.v, m); wa = smv(B.w, m); }
        if (kJacobi) sweep_jacobi<G, false>(frows, run_fast ? nr : 0, p.n_vel_iters, va, wa, gl);
        else if (waits_ok) {   // the row stream continues: rows from the start again
            rs.pf = 0;
            waits_ok = sweep_fast<G, false>(rs, total, trips, lam, va, wa, gl);
        }
        if (run_fast && gl == 0) { smv_set(B.v, m, va); smv_set(B.w, m, wa); }
        if (pf) sweep_env_pf<false>(p, E, S.row_base, frows, B, chunk_buf, lane, p.n_vel_iters);
        else if (valid && !fast && gl == 0) {
            if (kMulti && general_sm) sweep_general(rows, nr, p.n_vel_iters, ring, lam, B, false);
            else for (int it = 0; it < p.n_vel_iters; ++it) sweep(rows, nr, B, false);
        }
    }
    if (!waits_ok && lane == 0) atomicOr(p.status, kStatusTimeout);   // a row chunk never arrived
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

// ---------------------------------------------------------------------------------------
// Piles.  The prep (one block per pile env) applies the forces, places every pair's rows,
// colours the pairs greedily in pair order (each takes the lowest colour that no earlier
// pair sharing one of its movable bodies took; kMaxColors at most, the last gathering every
// pair left over) and hands the tables and the bodies' state to the sweep kernel (one
// cooperative launch over the GPU), which builds the rows (pile rows, the two-body fast
// form) and runs the Gauss-Seidel sweeps colour by colour.  The pairs of a colour share no
// movable body, so the warps solve them at once (a warp per pair, its rows in order) with
// exactly the updates of a sweep in colour order, pair order within a colour -- except the
// last colour, which one warp sweeps in pair order.  The prep's shared memory: the bodies
// (PileBodies), their colour masks and the pairs' tables (PileTables).

// exclusive prefix sum over the block (blockDim a multiple of 32, at most 1024); *total:
// the block's sum
__device__ int pile_scan(int v, int *warp_sums, int &total) {
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
        if (lane < nw) warp_sums[lane] = x;
    }
    __syncthreads();
    const int before = warp > 0 ? warp_sums[warp - 1] : 0;
    total = warp_sums[nw - 1];
    __syncthreads();
    return before + incl - v;
}

// Per-pair tables of the pile prep in shared memory (see pile_smem_bytes).
struct PileTables {
    unsigned *ab;             // local ids a | b << 16, bit 15 / 31 set when a / b is movable
    unsigned *rr;             // rows: start | count << 21 (within the pile's row region)
    unsigned short *order;    // the pairs with rows by colour (pair order within the last colour)
    unsigned char *col;       // colour, 254 before colouring, 255 without rows
};
constexpr unsigned kAbId = 0x3FFu;   // local ids are below kMaxPileBodies = 1024

constexpr int kPileThreads = 384;

// The greedy colouring of the pairs with rows, in pair order, by one warp: a batch of 32
// pairs is read into the lanes, then each pair of the batch in turn takes the lowest colour
// that neither of its movable bodies has taken yet (bodies' colour masks in shared memory;
// every lane computes the same colour, lane 0 updates the masks).
__device__ void pile_colour_warp(const PileTables &T, unsigned long long *used, int np, int lane) {
    for (int q0 = 0; q0 < np; q0 += 32) {
        const int q = q0 + lane;
        const bool has = q < np && T.col[q] != 255;
        const unsigned my_ab = has ? T.ab[q] : 0u;
        unsigned pend = __ballot_sync(0xffffffffu, has);
        int mine = 255;
        while (pend) {
            const int k = __ffs(pend) - 1;
            pend &= pend - 1;
            const unsigned abk = __shfl_sync(0xffffffffu, my_ab, k);
            const int a = (int)(abk & kAbId), b = (int)((abk >> 16) & kAbId);
            const unsigned long long ua = used[a], ub = used[b];   // zero for a body that never moves
            int c = __ffsll((long long)~(ua | ub)) - 1;
            if (c < 0 || c > kMaxColors - 1) c = kMaxColors - 1;
            if (lane == k) mine = c;
            __syncwarp();
            if (lane == 0) {
                if (abk & 0x8000u) used[a] = ua | (1ull << c);
                if (abk & 0x80000000u) used[b] = ub | (1ull << c);
            }
            __syncwarp();
        }
        if (has) T.col[q] = (unsigned char)mine;
    }
}

// The pile solve, part 1 (one block per pile): external forces, each pair's rows placed,
// the colours and the pairs by colour; hands the tables and the bodies' state to the sweep
// kernel through PileSolveMem.
__global__ void __launch_bounds__(kPileThreads, 1) pile_prep_kernel(SimParams p, const PileDev *piles,
                                                                     const int2 *counts, PileSolveMem M) {
    extern __shared__ __align__(16) float pile_smem[];
    __shared__ int warp_sums[32];
    __shared__ int cstart[kMaxColors + 1];
    __shared__ int fill[kMaxColors];
    __shared__ int s_colors;
    const PileDev P = piles[blockIdx.x];
    const int n = P.n_bodies, t = threadIdx.x, NT = blockDim.x;
    const int np = counts[blockIdx.x].x;
    PileBodies B;
    B.v = reinterpret_cast<float (*)[3]>(pile_smem);
    B.w = reinterpret_cast<float (*)[3]>(pile_smem + 3 * n);
    B.com = reinterpret_cast<float (*)[3]>(pile_smem + 6 * n);
    B.Iinv = reinterpret_cast<float (*)[6]>(pile_smem + 9 * n);
    B.invm = pile_smem + 15 * n;
    unsigned long long *used = reinterpret_cast<unsigned long long *>(pile_smem + 16 * n);   // 64 n bytes in
    PileTables T;
    T.ab = reinterpret_cast<unsigned *>(used + n);
    T.rr = T.ab + P.pcap;
    T.order = reinterpret_cast<unsigned short *>(T.rr + P.pcap);
    T.col = reinterpret_cast<unsigned char *>(T.order + P.pcap);
    unsigned char *mov = T.col + P.pcap;
    B.mov = mov;
    const float hs = p.hs;
    // 1. external forces
    for (int lb = t; lb < n; lb += NT) {
        body_forces(p, P.first_body + lb, lb, hs, B);
        const int ty = p.props[P.first_body + lb].type;
        mov[lb] = (ty == FW_BODY_DYNAMIC || ty == FW_BODY_FIXED_AXIS) ? 1 : 0;
        used[lb] = 0ull;
    }
    if (t < kMaxColors) fill[t] = 0;
    if (t == 0) s_colors = 0;
    __syncthreads();
    // 2. each pair's rows (its contacts, at most cap_pair) placed in pair order, rows past the
    // pile's row region dropped (overflow status); its bodies into the tables
    int base = 0;
    for (int c0 = 0; c0 < np; c0 += NT) {
        const int q = c0 + t;
        int nc = 0;
        if (q < np) {
            const int c = p.counts[P.pair0 + q];
            nc = c < p.cap_pair ? c : p.cap_pair;
        }
        int chunk;
        const int o = base + pile_scan(nc, warp_sums, chunk);
        if (q < np) {
            const int lo = o < P.rcap ? o : P.rcap, hi = o + nc < P.rcap ? o + nc : P.rcap;
            T.rr[q] = (unsigned)lo | ((unsigned)(hi - lo) << 21);
            T.col[q] = hi > lo ? 254 : 255;
            const PairDev &D = p.pairs[P.pair0 + q];
            const int a = D.local_a, b = D.local_b;
            T.ab[q] = (unsigned)a | (mov[a] ? 0x8000u : 0u) | ((unsigned)b << 16) | (mov[b] ? 0x80000000u : 0u);
        }
        base += chunk;
    }
    if (t == 0 && base > P.rcap) atomicOr(p.status, kStatusOverflow);
    __syncthreads();
    // 3. warp 0 colours the pairs (the sweep kernel builds the rows, on every SM)
    const int lane = t & 31, warp = t >> 5;
    if (warp == 0) pile_colour_warp(T, used, np, lane);
    __syncthreads();
    // 4. the pairs by colour: counts, starts, then each pair a slot in its colour (any order
    // within a colour gives the same sweep: its pairs share no movable body)
    for (int q = t; q < np; q += NT) {
        const int c = T.col[q];
        if (c != 255) {
            atomicAdd(&fill[c], 1);
            atomicMax(&s_colors, c + 1);
        }
        M.color[P.pair0 + q] = (unsigned char)c;
        M.ab[P.pair0 + q] = T.ab[q];
        M.rr[P.pair0 + q] = T.rr[q];
    }
    __syncthreads();
    if (t == 0) {
        cstart[0] = 0;
        for (int c = 0; c < kMaxColors; ++c) {
            cstart[c + 1] = cstart[c] + fill[c];
            fill[c] = cstart[c];
        }
    }
    __syncthreads();
    for (int q = t; q < np; q += NT) {
        const int c = T.col[q];
        if (c != 255 && c != kMaxColors - 1) M.order[P.pair0 + atomicAdd(&fill[c], 1)] = q;
    }
    // the last colour's pairs may share bodies: one warp sweeps them, in pair order
    if (t == 0 && s_colors == kMaxColors) {
        int k = cstart[kMaxColors - 1];
        for (int q = 0; q < np; ++q)
            if (T.col[q] == kMaxColors - 1) M.order[P.pair0 + k++] = q;
    }
    for (int c = t; c <= kMaxColors; c += NT) M.cstart[blockIdx.x * (kMaxColors + 1) + c] = cstart[c];
    if (t == 0) M.ncol[blockIdx.x] = s_colors;
    // 5. the bodies' state after the forces, for the sweeps
    for (int lb = t; lb < n; lb += NT) {
        const int bi = P.first_body + lb;
        M.bv[bi] = make_float4(B.v[lb][0], B.v[lb][1], B.v[lb][2], B.invm[lb]);
        M.bw[bi] = make_float4(B.w[lb][0], B.w[lb][1], B.w[lb][2], mov[lb] ? 1.0f : 0.0f);
        M.bcom[bi] = make_float4(B.com[lb][0], B.com[lb][1], B.com[lb][2], 0.0f);
        M.binv[2 * bi] = make_float4(B.Iinv[lb][0], B.Iinv[lb][1], B.Iinv[lb][2], B.Iinv[lb][3]);
        M.binv[2 * bi + 1] = make_float4(B.Iinv[lb][4], B.Iinv[lb][5], 0.0f, 0.0f);
    }
}

// ---- the pile solve, part 2: one cooperative kernel over the whole GPU
constexpr int kSweepWarps = 8;                      // warps per block of the sweep kernel
constexpr int kSweepChunk = 16;                     // rows per shared-memory chunk of a pair
constexpr int kSweepBufF4 = 2 * kSweepChunk * kPileRowF4;   // two chunks per warp
constexpr int kGridWaitTries = 1 << 20;             // bounded grid-barrier polls (about a second)

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *a) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(a) : "memory");
    return v;
}
__device__ __forceinline__ float4 ldcg4(const float4 *a) { return __ldcg(a); }

// Barrier of every block of the (cooperative) launch: block barrier, then thread 0 makes
// the block's writes visible at device scope, arrives and waits (bounded) until `target`
// blocks have arrived.  A wait that gives up sets the timeout status; the block then stops
// waiting at later barriers (it only arrives), so that the launch always ends.
__device__ void grid_barrier(unsigned *bar, unsigned target, unsigned *status, int *dead) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        if (!*dead) {
            int tries = 0;
            while (ld_acquire_gpu(bar) < target) {
                if (++tries > kGridWaitTries) {
                    atomicOr(status, kStatusTimeout);
                    *dead = 1;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// A pile row as one lane of a pair's warp holds it: its quarter's part of the scaled
// Jacobian (PfJ; formed into the scaled velocities one step before the row is solved), its
// quarter's update vectors, the couplings and the impulse word (PfCW).
struct PfJ {
    float4 j[3];
};
struct PfCW {
    float4 c[3];
    float4 w[3];
    float4 l;
};
__device__ __forceinline__ void read_pf_j(unsigned row, unsigned qo, PfJ &r) {
#pragma unroll
    for (int k = 0; k < 3; ++k) r.j[k] = lds4(row + qo + 16u * k);
}
__device__ __forceinline__ void read_pf_cw(unsigned row, unsigned qo, PfCW &r) {
#pragma unroll
    for (int k = 0; k < 3; ++k) r.w[k] = lds4(row + qo + 16u * (3 + k));
#pragma unroll
    for (int k = 0; k < 3; ++k) r.c[k] = lds4(row + 16u * (kPfC + k));
    r.l = lds4(row + 16u * kPfL);
}
// scaled velocities of a pile row at the velocity u: each lane dots its quarter, the four
// lanes of the quarter group sum the parts (xor 1, then xor 2: the same sum on all four)
template <bool kBias>
__device__ __forceinline__ void pf_base(const PfJ &g, V3 u, float &bn, float &b1, float &b2) {
    float pn = __fmaf_rn(g.j[0].z, u.z, __fmaf_rn(g.j[0].y, u.y, __fmaf_rn(g.j[0].x, u.x, kBias ? g.j[0].w : 0.0f)));
    float p1 = __fmaf_rn(g.j[1].z, u.z, __fmaf_rn(g.j[1].y, u.y, __fmaf_rn(g.j[1].x, u.x, g.j[1].w)));
    float p2 = __fmaf_rn(g.j[2].z, u.z, __fmaf_rn(g.j[2].y, u.y, __fmaf_rn(g.j[2].x, u.x, g.j[2].w)));
    pn += __shfl_xor_sync(0xffffffffu, pn, 1);
    p1 += __shfl_xor_sync(0xffffffffu, p1, 1);
    p2 += __shfl_xor_sync(0xffffffffu, p2, 1);
    bn = pn + __shfl_xor_sync(0xffffffffu, pn, 2);
    b1 = p1 + __shfl_xor_sync(0xffffffffu, p1, 2);
    b2 = p2 + __shfl_xor_sync(0xffffffffu, p2, 2);
}
// One Gauss-Seidel step of a pile pair, pipelined over three rows as gs_step: row j (f) is
// solved from its carried scaled velocities while row j + 1's scaled velocities are formed
// from its Jacobian part jn at the velocity before row j and the loads of row j + 1 (fn,
// shared address rn) and row j + 2's Jacobian part (jnn, at rnn) are issued.  Lane 0
// writes the new impulse word to the row in global memory (lam).
template <bool kBias>
__device__ __forceinline__ void pf_step(const PfCW &f, const PfJ &jn, PfCW &fn, PfJ &jnn, SweepRegs &st,
                                        unsigned rn, unsigned rnn, unsigned qo, float4 *lam, bool leader) {
    float bn, b1, b2;
    pf_base<kBias>(jn, st.u, bn, b1, b2);
    read_pf_cw(rn, qo, fn);
    read_pf_j(rnn, qo, jnn);
    const float4 L = f.l;
    const float dl = fmaxf(st.sn, -L.x);                  // lambda_n' - lambda_n
    const V3 u = st.u;
    const V3 ud = v3(__fmaf_rn(dl, f.w[0].x, u.x), __fmaf_rn(dl, f.w[0].y, u.y), __fmaf_rn(dl, f.w[0].z, u.z));
    const float xn = __fmaf_rn(f.c[0].w, dl, bn), x1 = __fmaf_rn(f.c[1].z, dl, b1), x2 = __fmaf_rn(f.c[2].y, dl, b2);
    const float ln = L.x + dl;
    const float t1 = __fmaf_rn(f.c[0].x, dl, st.s1 + L.y);
    const float t2 = __fmaf_rn(f.c[0].y, dl, st.s2 + L.z);
    const float sc = fminf(1.0f, (f.c[0].z * ln) * rsqrtf(__fmaf_rn(t1, t1, t2 * t2)));
    const float e1 = __fmaf_rn(t1, sc, -L.y), e2 = __fmaf_rn(t2, sc, -L.z);
    st.sn = __fmaf_rn(f.c[1].y, e2, __fmaf_rn(f.c[1].x, e1, xn));
    st.s1 = __fmaf_rn(f.c[2].x, e2, __fmaf_rn(f.c[1].w, e1, x1));
    st.s2 = __fmaf_rn(f.c[2].w, e2, __fmaf_rn(f.c[2].z, e1, x2));
    st.u = v3(__fmaf_rn(e2, f.w[2].x, __fmaf_rn(e1, f.w[1].x, ud.x)),
              __fmaf_rn(e2, f.w[2].y, __fmaf_rn(e1, f.w[1].y, ud.y)),
              __fmaf_rn(e2, f.w[2].z, __fmaf_rn(e1, f.w[1].z, ud.z)));
    if (leader) __stcg(lam, make_float4(ln, L.y + e1, L.z + e2, 0.0f));
}

// Chunk ch of a pair's n rows (kCh rows per chunk) into the warp's buffer (ch & 1), by all 32
// lanes (one commit group).
template <int kCh>
__device__ __forceinline__ void pf_issue_chunk(const float4 *rows, int n, int ch, float4 *buf, int lane) {
    constexpr int kChF4 = kCh * kPileRowF4;
    const int rows_in = min(kCh, n - ch * kCh);
    float4 *dst = buf + (ch & 1) * kChF4;
    const float4 *s0 = rows + (size_t)ch * kChF4;
    for (int k = lane; k < rows_in * kPileRowF4; k += 32) cp_async16(dst + k, s0 + k);
    cp_async_commit();
}
// The first two chunks of a pair (the start of pf_pair_rows), issued ahead of it.
template <int kCh>
__device__ __forceinline__ void pf_prefetch(const float4 *rows, int n, float4 *buf, int lane) {
    pf_issue_chunk<kCh>(rows, n, 0, buf, lane);
    if (n > kCh) pf_issue_chunk<kCh>(rows, n, 1, buf, lane);
}

// The rows 0 .. n - 1 (global, kPileRowF4 float4 each) of one pair, by one warp, from the
// velocity quarter u of this lane (lane & 3, see build_pile_row; the other groups of four
// lanes repeat the first's work), which it leaves as the pair's Gauss-Seidel update makes
// it.  The lanes stream the rows through two shared-memory chunks of kCh rows at buf
// (cp.async, L2 only: impulses may have been written by other SMs; chunk c + 1 is waited
// for at step kCh c + kCh - 2, whose loads reach its first row, and chunk c + 2 issued into
// chunk c's buffer after it); lane 0 writes each impulse word back.  prefetched: the first
// chunks were issued by pf_prefetch.  Called by all 32 lanes.
template <bool kBias, int kCh>
__device__ void pf_pair_rows(float4 *rows, int n, float4 *buf, int lane, V3 &u, bool prefetched) {
    constexpr int kChF4 = kCh * kPileRowF4;
    const int q = lane & 3;
    SweepRegs st;
    st.u = u;
    const int nch = (n + kCh - 1) / kCh;
    auto issue = [&](int ch) { pf_issue_chunk<kCh>(rows, n, ch, buf, lane); };
    if (!prefetched) pf_prefetch<kCh>(rows, n, buf, lane);
    if (nch > 1) {
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    __syncwarp();
    const unsigned b0 = smem_addr(buf), qo = 16u * kPfQ * q;
    constexpr unsigned kRowBP = 16u * kPileRowF4, kChunkBP = 16u * kChF4;
    // prologue: row 0's words and scaled velocities, row 1's Jacobian part (rows past n are
    // read from the buffers but never used)
    PfCW A, B;
    PfJ JA, JB;
    read_pf_cw(b0, qo, A);
    read_pf_j(b0, qo, JA);
    pf_base<kBias>(JA, st.u, st.sn, st.s1, st.s2);
    read_pf_j(b0 + kRowBP, qo, JB);
    const bool leader = lane == 0;
    // chunk c (buffer cur; chunk c + 1 in nxt) row by row, two steps per trip at constant
    // shared-memory offsets; step kCh - 2 of the chunk loads the next chunk's first row: it
    // waits for that chunk, and after it chunk c's buffer takes chunk c + 2.  A full chunk
    // runs as one straight-line block of steps (step guards would split every step into its
    // own block: measured slower), the last partial one stops at row n.
    for (int c = 0; c < nch; ++c) {
        const unsigned cur = b0 + kChunkBP * (unsigned)(c & 1), nxt = b0 + kChunkBP * (unsigned)((c + 1) & 1);
        float4 *lam = rows + (size_t)kChF4 * c + kPfL;
        const int left = n - kCh * c;   // rows of this chunk and after
        if (left >= kCh) {
#pragma unroll
            for (int jj = 0; jj < kCh; jj += 2) {
                if (jj == kCh - 2 && c + 1 < nch) {
                    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
                    __syncwarp();
                }
                const unsigned r1 = (jj + 1 < kCh) ? cur + kRowBP * (jj + 1) : nxt + kRowBP * (jj + 1 - kCh);
                const unsigned r2 = (jj + 2 < kCh) ? cur + kRowBP * (jj + 2) : nxt + kRowBP * (jj + 2 - kCh);
                const unsigned r3 = (jj + 3 < kCh) ? cur + kRowBP * (jj + 3) : nxt + kRowBP * (jj + 3 - kCh);
                pf_step<kBias>(A, JB, B, JA, st, r1, r2, qo, lam + kPileRowF4 * jj, leader);
                if (jj == kCh - 2 && c + 2 < nch) {
                    __syncwarp();
                    issue(c + 2);
                }
                pf_step<kBias>(B, JA, A, JB, st, r2, r3, qo, lam + kPileRowF4 * (jj + 1), leader);
            }
        } else {   // the pair's last, partial chunk (no next chunk to wait for or to issue)
#pragma unroll
            for (int jj = 0; jj < kCh; jj += 2) {
                if (jj >= left) break;
                // rows past the chunk (read, never used) wrap into the other buffer: in bounds
                const unsigned r1 = (jj + 1 < kCh) ? cur + kRowBP * (jj + 1) : nxt + kRowBP * (jj + 1 - kCh);
                const unsigned r2 = (jj + 2 < kCh) ? cur + kRowBP * (jj + 2) : nxt + kRowBP * (jj + 2 - kCh);
                const unsigned r3 = (jj + 3 < kCh) ? cur + kRowBP * (jj + 3) : nxt + kRowBP * (jj + 3 - kCh);
                pf_step<kBias>(A, JB, B, JA, st, r1, r2, qo, lam + kPileRowF4 * jj, leader);
                if (jj + 1 >= left) break;
                pf_step<kBias>(B, JA, A, JB, st, r2, r3, qo, lam + kPileRowF4 * (jj + 1), leader);
            }
        }
    }
    // (every chunk issued was waited for: chunk c at step kCh (c - 1) + kCh - 2 < n)
    u = st.u;
}

// n_sweeps Gauss-Seidel sweeps of an env of several movable bodies over its two-body fast
// rows, pair by pair in pair order (the order of the general form's sweep): the lanes take
// the pair's velocity quarters from the env's body store, pf_pair_rows runs its rows, lanes
// 0-3 write the quarters back before the next pair (which may share a body) reads them.
// One env per warp: all 32 lanes take the same pairs.
template <bool kBias>
__device__ void sweep_env_pf(const SimParams &p, const EnvDev &E, const int *row_base, float4 *frows, BodySm &B,
                             float4 *buf, int lane, int n_sweeps) {
    const int q = lane & 3;
    for (int it = 0; it < n_sweeps; ++it)
        for (int k = 0; k < E.n_pairs; ++k) {
            const int r0 = row_base[k], n = row_base[k + 1] - r0;
            if (n == 0) continue;
            const PairDev P = p.pairs[E.first_pair + k];
            const int bi = q < 2 ? P.local_a : P.local_b;
            V3 u = (q & 1) ? smv(B.w, bi) : smv(B.v, bi);
            pf_pair_rows<kBias, kEnvPfChunk>(frows + (size_t)kPileRowF4 * r0, n, buf, lane, u, false);
            __syncwarp();
            if (lane < 4) {
                if (q & 1) smv_set(B.w, bi, u);
                else smv_set(B.v, bi, u);
            }
            __syncwarp();
        }
}

__device__ __forceinline__ void pile_prefetch(const float4 *rows, int n, float4 *buf, int lane) {
    pf_prefetch<kSweepChunk>(rows, n, buf, lane);
}

// One pile pair between global bodies ga, gb (pf_pair_rows with kSweepChunk-row chunks):
// the lane's velocity quarter comes from global memory (L2: other SMs wrote it) and goes
// back there at the end (movable bodies only).
template <bool kBias>
__device__ void sweep_pair_warp(float4 *rows, int n, int ga, int gb, float4 *buf, const PileSolveMem &M, int lane,
                                bool prefetched) {
    const int q = lane & 3;
    const int gi = q < 2 ? ga : gb;
    const float4 bv = ldcg4(M.bv + gi), bw = ldcg4(M.bw + gi);
    V3 u = (q & 1) ? v3(bw.x, bw.y, bw.z) : v3(bv.x, bv.y, bv.z);
    pf_pair_rows<kBias, kSweepChunk>(rows, n, buf, lane, u, prefetched);
    if (lane < 4 && bw.w != 0.0f) {
        if (q & 1) M.bw[gi] = make_float4(u.x, u.y, u.z, bw.w);
        else M.bv[gi] = make_float4(u.x, u.y, u.z, bv.w);
    }
    __syncwarp();
}

// A warp's first pair in each colour but the last (PileWork: row index, rows, bodies a, b
// (global ids); rows = 0: none), and a bit per colour in which it has more pairs: built once
// per launch, so that a colour's turn starts without the dependent loads of the tables.
constexpr int kWorkColors = kMaxColors - 1;
struct PileWarpWork {
    int4 first[kWorkColors];
    unsigned long long more;
};
__device__ void pile_warp_work(const PileSolveMem &M, const PileDev *piles, int n_piles, int n_colors, int gw, int W,
                               int lane, PileWarpWork &ww) {
    unsigned long long more = 0ull;
    for (int c = lane; c < n_colors && c < kWorkColors; c += 32) {
        int4 e = make_int4(0, 0, 0, 0);
        bool found = false, again = false;
        for (int k0 = 0; k0 < n_piles && !again; ++k0) {
            const PileDev &P = piles[k0];
            const int *cs = M.cstart + k0 * (kMaxColors + 1);
            for (int k = cs[c] + gw; k < cs[c + 1]; k += W) {
                if (found) { again = true; break; }
                const int q = M.order[P.pair0 + k];
                const unsigned ab = M.ab[P.pair0 + q], rr = M.rr[P.pair0 + q];
                e = make_int4(P.row0 + (int)(rr & (kPileMaxRows - 1)), (int)(rr >> 21),
                              P.first_body + (int)(ab & kAbId), P.first_body + (int)((ab >> 16) & kAbId));
                found = true;
            }
        }
        ww.first[c] = e;
        if (again) more |= 1ull << c;
    }
    more = __reduce_or_sync(0xffffffffu, (unsigned)more) | ((unsigned long long)__reduce_or_sync(0xffffffffu, (unsigned)(more >> 32)) << 32);
    if (lane == 0) ww.more = more;
    __syncwarp();
}

// n_sweeps Gauss-Seidel sweeps over every pile, colour by colour with a grid barrier after
// each colour: within a colour the launch's warps take the pairs (any order: they share no
// movable body); the last colour, whose pairs may share bodies, is swept by warp 0 of the
// launch in pair order.  A warp's first pair of a colour comes from its PileWarpWork; a
// pair's rows (and impulses) do not change between its colour's turns, only the bodies'
// velocities do, so before each barrier the warp issues the first chunks of its pair of the
// next colour (with one colour, that pair may be the one just swept: no prefetch).
template <bool kBias>
__device__ void pile_sweep_passes(const SimParams &p, const PileDev *piles, int n_piles, const PileSolveMem &M,
                                  float4 *rows, float4 *buf, const PileWarpWork &ww, int n_colors, int n_sweeps,
                                  unsigned &nbar, int *dead) {
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kSweepWarps + (threadIdx.x >> 5), W = gridDim.x * kSweepWarps;
    bool pre = false;   // the first pair of the coming colour prefetched
    for (int it = 0; it < n_sweeps; ++it) {
        for (int c = 0; c < n_colors; ++c) {
            const bool serial = c == kMaxColors - 1;
            if (!serial) {
                const int4 e = ww.first[c];
                if (e.y > 0)
                    sweep_pair_warp<kBias>(rows + (size_t)kPileRowF4 * e.x, e.y, e.z, e.w, buf, M, lane, pre);
            }
            if (serial || ((ww.more >> c) & 1ull)) {   // the rest (the last colour: warp 0 alone)
                const int skip = serial ? -1 : ww.first[c].x;
                for (int k0 = 0; k0 < n_piles; ++k0) {
                    const PileDev &P = piles[k0];
                    const int *cs = M.cstart + k0 * (kMaxColors + 1);
                    const int b = cs[c], e = cs[c + 1];
                    if (serial && gw != 0) continue;
                    for (int k = b + (serial ? 0 : gw); k < e; k += serial ? 1 : W) {
                        const int q = M.order[P.pair0 + k];
                        const unsigned ab = M.ab[P.pair0 + q], rr = M.rr[P.pair0 + q];
                        const int r0 = P.row0 + (int)(rr & (kPileMaxRows - 1)), nr = (int)(rr >> 21);
                        if (r0 == skip) continue;
                        sweep_pair_warp<kBias>(rows + (size_t)kPileRowF4 * r0, nr, P.first_body + (int)(ab & kAbId),
                                               P.first_body + (int)((ab >> 16) & kAbId), buf, M, lane, false);
                    }
                }
            }
            // the next colour's first pair (none after the passes' last colour)
            const int cn = c + 1 < n_colors ? c + 1 : 0;
            pre = false;
            if (n_colors > 1 && (c + 1 < n_colors || it + 1 < n_sweeps) && cn != kMaxColors - 1 && ww.first[cn].y > 0) {
                pile_prefetch(rows + (size_t)kPileRowF4 * ww.first[cn].x, ww.first[cn].y, buf, lane);
                pre = true;
            }
            ++nbar;
            grid_barrier(M.bar, nbar * gridDim.x + (p.stall == 1 ? 1u : 0u), p.status, dead);
        }
    }
}

__global__ void __launch_bounds__(kSweepWarps * 32, 1) pile_sweep_kernel(SimParams p, const PileDev *piles,
                                                                          int n_piles, PileSolveMem M, float4 *rows) {
    extern __shared__ __align__(16) float4 sweep_smem[];
    __shared__ int dead;
    if (threadIdx.x == 0) dead = 0;
    __syncthreads();
    float4 *buf = sweep_smem + (threadIdx.x >> 5) * kSweepBufF4;
    int n_colors = 0;
    for (int k = 0; k < n_piles; ++k) n_colors = max(n_colors, M.ncol[k]);
    unsigned nbar = 0;
    const float hs = p.hs;
    // 4. each pair's rows, a warp per pair with rows (the pairs in colour order), its lanes
    // over the pair's contacts; then the couplings between the pair's neighbouring rows
    {
        const int lane = threadIdx.x & 31;
        const int gw = blockIdx.x * kSweepWarps + (threadIdx.x >> 5), W = gridDim.x * kSweepWarps;
        for (int k0 = 0; k0 < n_piles; ++k0) {
            const PileDev &P = piles[k0];
            const int total = M.cstart[k0 * (kMaxColors + 1) + kMaxColors];
            for (int k = gw; k < total; k += W) {
                const int q = M.order[P.pair0 + k];
                const unsigned ab = M.ab[P.pair0 + q], rr = M.rr[P.pair0 + q];
                const int r0 = (int)(rr & (kPileMaxRows - 1)), cnt = (int)(rr >> 21);
                const int a = P.first_body + (int)(ab & kAbId), b = P.first_body + (int)((ab >> 16) & kAbId);
                const float4 ca = M.bcom[a], cb = M.bcom[b], ia0 = M.binv[2 * a], ia1 = M.binv[2 * a + 1];
                const float4 ib0 = M.binv[2 * b], ib1 = M.binv[2 * b + 1];
                const float Ia[6] = {ia0.x, ia0.y, ia0.z, ia0.w, ia1.x, ia1.y};
                const float Ib[6] = {ib0.x, ib0.y, ib0.z, ib0.w, ib1.x, ib1.y};
                const float ima = M.bv[a].w, imb = M.bv[b].w;
                const float mu = p.pairs[P.pair0 + q].mu;
                const DContact *con = p.contacts + (size_t)(P.pair0 + q) * p.cap_pair;
                float4 *pr = rows + (size_t)kPileRowF4 * (P.row0 + r0);
                for (int i = lane; i < cnt; i += 32)
                    build_pile_row(pr + kPileRowF4 * i, con[i], v3(ca.x, ca.y, ca.z), v3(cb.x, cb.y, cb.z), Ia, Ib,
                                   ima, imb, mu, hs, p.baumgarte);
                __syncwarp();   // the pair's rows (global) written before other lanes read them
                for (int i = lane; i < cnt; i += 32)
                    couple_pile_row(pr + kPileRowF4 * i, i + 1 < cnt ? pr + kPileRowF4 * (i + 1) : nullptr);
                __syncwarp();
            }
        }
    }
    __shared__ PileWarpWork s_work[kSweepWarps];
    PileWarpWork &ww = s_work[threadIdx.x >> 5];
    pile_warp_work(M, piles, n_piles, n_colors, blockIdx.x * kSweepWarps + (threadIdx.x >> 5),
                   gridDim.x * kSweepWarps, threadIdx.x & 31, ww);
    ++nbar;
    grid_barrier(M.bar, nbar * gridDim.x + (p.stall == 1 ? 1u : 0u), p.status, &dead);
    // 5. Gauss-Seidel sweeps
    pile_sweep_passes<true>(p, piles, n_piles, M, rows, buf, ww, n_colors, p.n_iters, nbar, &dead);
    // 6. integration, a thread per body
    const int gt = blockIdx.x * blockDim.x + threadIdx.x, GT = gridDim.x * blockDim.x;
    for (int k = 0; k < n_piles; ++k) {
        const PileDev &P = piles[k];
        for (int lb = gt; lb < P.n_bodies; lb += GT) {
            const int bi = P.first_body + lb;
            const BodyProps Pb = p.props[bi];
            const float4 v4 = ldcg4(M.bv + bi), w4 = ldcg4(M.bw + bi), c4 = ldcg4(M.bcom + bi);
            V3 w = v3(w4.x, w4.y, w4.z);
            const float4 q = integrate_core(p, Pb, bi, hs, w, v3(v4.x, v4.y, v4.z), v3(c4.x, c4.y, c4.z));
            p.quat[4 * bi] = q.x; p.quat[4 * bi + 1] = q.y; p.quat[4 * bi + 2] = q.z; p.quat[4 * bi + 3] = q.w;
            if (Pb.type != FW_BODY_STATIC) M.bw[bi] = make_float4(w.x, w.y, w.z, w4.w);
        }
    }
    ++nbar;
    grid_barrier(M.bar, nbar * gridDim.x + (p.stall == 1 ? 1u : 0u), p.status, &dead);
    // 7. optional bias-free sweeps
    if (p.n_vel_iters > 0)
        pile_sweep_passes<false>(p, piles, n_piles, M, rows, buf, ww, n_colors, p.n_vel_iters, nbar, &dead);
    for (int k = 0; k < n_piles; ++k) {
        const PileDev &P = piles[k];
        for (int lb = gt; lb < P.n_bodies; lb += GT) {
            const int bi = P.first_body + lb;
            const float4 v4 = ldcg4(M.bv + bi), w4 = ldcg4(M.bw + bi);
            const V3 v = v3(v4.x, v4.y, v4.z), w = v3(w4.x, w4.y, w4.z);
            st3(p.linvel + 3 * bi, v);
            st3(p.angvel + 3 * bi, w);
            if (!(isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(w.x) && isfinite(w.y) && isfinite(w.z)))
                atomicOr(p.status, kStatusNonFinite);
        }
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

size_t pile_smem_bytes(int n_bodies, int pcap) {
    // bodies (16 floats, a colour mask, a movable flag); per pair its bodies, its rows, an
    // order slot and a colour (PileTables)
    return (size_t)n_bodies * (16 * sizeof(float) + sizeof(unsigned long long) + 1) + (size_t)pcap * 11 + 16;
}

cudaError_t prepare_pile_solve(int optin, int device, int *max_dyn, int *sweep_blocks) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, pile_prep_kernel);
    if (e != cudaSuccess) return e;
    *max_dyn = optin - (int)a.sharedSizeBytes;
    e = cudaFuncSetAttribute(pile_prep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, *max_dyn);
    if (e != cudaSuccess) return e;
    const int smem = kSweepWarps * kSweepBufF4 * (int)sizeof(float4);
    e = cudaFuncSetAttribute(pile_sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0, n_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pile_sweep_kernel, kSweepWarps * 32, smem);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return e;
    // one block per SM (eight warps each: more warps than any colour of a 1,024-body pile has
    // pairs), every block resident at once (the launch is cooperative); fewer blocks make the
    // grid barriers cheaper
    *sweep_blocks = per_sm * n_sm;
    return *sweep_blocks > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

cudaError_t launch_pile_solve(const SimParams &p, const PileDev *piles, int n_piles, const int2 *counts,
                              const PileSolveMem &m, float4 *rows, size_t smem, int sweep_blocks, cudaStream_t s) {
    if (n_piles <= 0) return cudaSuccess;
    pile_prep_kernel<<<n_piles, kPileThreads, smem, s>>>(p, piles, counts, m);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(m.bar, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(sweep_blocks);
    cfg.blockDim = dim3(kSweepWarps * 32);
    cfg.dynamicSmemBytes = kSweepWarps * kSweepBufF4 * sizeof(float4);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, pile_sweep_kernel, p, piles, n_piles, m, rows);
}

template <int kGroups>
static cudaError_t prepare_one(int optin, int *max_dyn) {
    void (*const k[3])(SimParams) = {solve_kernel<kGroups, kVarGS>, solve_kernel<kGroups, kVarMulti>,
                                     solve_kernel<kGroups, kVarJacobi>};
    size_t stat = 0;
    for (int v = 0; v < 3; ++v) {
        cudaFuncAttributes a;
        cudaError_t e = cudaFuncGetAttributes(&a, k[v]);
        if (e != cudaSuccess) return e;
        if (a.sharedSizeBytes > stat) stat = a.sharedSizeBytes;
    }
    *max_dyn = optin - (int)stat;
    for (int v = 0; v < 3; ++v) {
        cudaError_t e = cudaFuncSetAttribute(k[v], cudaFuncAttributeMaxDynamicSharedMemorySize, *max_dyn);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <int kGroups>
static void launch_variant(const SimParams &p, dim3 grid, dim3 block, size_t smem, cudaStream_t s) {
    if (p.solver == 1) solve_kernel<kGroups, kVarJacobi><<<grid, block, smem, s>>>(p);
    else if (p.multi_movable) solve_kernel<kGroups, kVarMulti><<<grid, block, smem, s>>>(p);
    else solve_kernel<kGroups, kVarGS><<<grid, block, smem, s>>>(p);
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
    const dim3 grid(blocks), block(32 * sh.warps);
    if (sh.groups == 1) launch_variant<1>(p, grid, block, sh.smem, s);
    else if (sh.groups == 2) launch_variant<2>(p, grid, block, sh.smem, s);
    else if (sh.groups == 4) launch_variant<4>(p, grid, block, sh.smem, s);
    else launch_variant<8>(p, grid, block, sh.smem, s);
    return cudaGetLastError();
}

}  // namespace fw
