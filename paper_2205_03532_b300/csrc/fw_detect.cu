// fw_detect.cu -- SDF narrow phase fused with contact reduction (Sec. III-A, III-C,
// Algorithm 1).  One CTA per shape pair; the pair's Generate batches of 1024 samples are
// queried, compacted in sample order into shared memory, assigned to existing patches,
// and the rest turned into new patches (FindDeepest / BinReduce / AddPatch).  Patches
// live in shared memory for the whole pair; only the reduced contacts reach global
// memory, plus the data of slot winners in a per-sample scratch line.
#include "fw_device.cuh"

namespace fw {

namespace {

constexpr int kT = kDetectThreads;
constexpr int kPerThread = kBatch / kT;   // 4
constexpr unsigned long long kNoKey = ~0ull;

__constant__ float c_cos6[6] = {1.0f, 0.5f, -0.5f, -1.0f, -0.5f, 0.5f};
__constant__ float c_sin6[6] = {0.0f, 0.8660254037844386f, 0.8660254037844386f, 0.0f,
                                -0.8660254037844386f, -0.8660254037844386f};

// Shared-memory layout (dynamic).  NP = max_patches + 1 (the last slot is the patch being
// built by the while loop).
struct Smem {
    float *cx, *cy, *cz, *cnx, *cny, *cnz, *cphi;
    int *cidx;
    short *cst;                 // -1 unassigned, -2 joining a new patch, -3 consumed, >= 0 patch id
    float *pn, *pa, *pt1, *pt2; // 3 x NP each, component-major
    unsigned long long *keys;   // kSlots x NP
    int *misc;                  // [0] n_cand, [1] n_patches, [2..9] warp counts
};

__device__ __forceinline__ Smem carve(unsigned char *base, int NP) {
    Smem s;
    float *f = reinterpret_cast<float *>(base);
    s.cx = f; s.cy = f + kBatch; s.cz = f + 2 * kBatch;
    s.cnx = f + 3 * kBatch; s.cny = f + 4 * kBatch; s.cnz = f + 5 * kBatch; s.cphi = f + 6 * kBatch;
    s.cidx = reinterpret_cast<int *>(f + 7 * kBatch);
    unsigned long long *k = reinterpret_cast<unsigned long long *>(f + 8 * kBatch);
    s.keys = k;
    float *pf = reinterpret_cast<float *>(k + kSlots * NP);
    s.pn = pf; s.pa = pf + 3 * NP; s.pt1 = pf + 6 * NP; s.pt2 = pf + 9 * NP;
    s.cst = reinterpret_cast<short *>(pf + 12 * NP);
    s.misc = reinterpret_cast<int *>(s.cst + kBatch);
    return s;
}

__host__ __device__ inline size_t smem_bytes(int NP) {
    return (size_t)8 * kBatch * 4 + (size_t)kSlots * NP * 8 + (size_t)12 * NP * 4 + (size_t)kBatch * 2 +
           16 * 4;
}

// Per-pair transform, computed once per CTA.
struct PairXf {
    M3 RA, RB;
    V3 pA, pB;
};

__device__ __forceinline__ void load_pose(const SimParams &p, int body, M3 &R, V3 &t) {
    float4 q = make_float4(p.quat[4 * body], p.quat[4 * body + 1], p.quat[4 * body + 2], p.quat[4 * body + 3]);
    R = quat_to_mat(q);
    t = ld3(p.pos + 3 * body);
}

// The narrow phase of one sample: world point, world normal and signed distance.
// Returns false when the point is outside the SDF grid or the gradient vanishes.
__device__ __forceinline__ bool query_sample(const PairXf &X, const AssetDev &gb, float4 s, V3 &xw,
                                             V3 &nw, float &phi) {
    xw = mul(X.RA, v3(s.x, s.y, s.z)) + X.pA;
    V3 xb = mul_t(X.RB, xw - X.pB);
    V3 g;
    if (!sdf_lookup_any(gb, xb, phi, g)) return false;
    float gg = dot(g, g);
    if (!(gg >= 1e-24f)) return false;          // |grad| < 1e-12 makes no candidate
    V3 nb = (1.0f / sqrtf(gg)) * g;
    nw = mul(X.RB, nb);
    return true;
}

__device__ __forceinline__ unsigned long long slot_key(float score, int sample) {
    return ((unsigned long long)ord_f32(score) << 32) | (unsigned)(0xFFFFFFFFu - (unsigned)sample);
}

// score of candidate (x, phi) for slot s of the patch with anchor a and basis t1, t2
__device__ __forceinline__ float slot_score(int s, V3 x, float phi, V3 a, V3 t1, V3 t2) {
    if (s == 0) return -phi;
    V3 d = x - a;
    float p1 = dot(d, t1), p2 = dot(d, t2);
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

__device__ __forceinline__ int key_sample(unsigned long long k) {
    return (int)(0xFFFFFFFFu - (unsigned)(k & 0xFFFFFFFFull));
}

// M = -phi_deepest + sqrt(area of the polygon through the distinct direction-slot
// points, in slot order, in the patch plane).  Reads winners' data from scratch.
__device__ float patch_measure(const Smem &S, int NP, int j, const float4 *scr) {
    const int deep = key_sample(S.keys[j]);
    float phid = scr[2 * deep].w;
    V3 a = pvec(S.pa, NP, j), t1 = pvec(S.pt1, NP, j), t2 = pvec(S.pt2, NP, j);
    float xs[6], ys[6];
    int seen[6], n = 0;
    for (int s = 1; s < kSlots; ++s) {
        const int id = key_sample(S.keys[s * NP + j]);
        bool dup = false;
        for (int t = 0; t < n; ++t) dup |= (seen[t] == id);
        if (dup) continue;
        float4 q = scr[2 * id];
        V3 d = v3(q.x, q.y, q.z) - a;
        xs[n] = dot(d, t1);
        ys[n] = dot(d, t2);
        seen[n++] = id;
    }
    float area2 = 0.0f;
    for (int i = 0; i < n; ++i) {
        int k = (i + 1 == n) ? 0 : i + 1;
        area2 += xs[i] * ys[k] - xs[k] * ys[i];
    }
    return -phid + sqrtf(0.5f * fabsf(area2));
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = (w < v) ? w : v;
    }
    return v;
}
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = (w > v) ? w : v;
    }
    return v;
}

// Algorithm 1 body for one batch whose candidates are in shared memory (S.misc[0] of
// them, in sample order).  Patches persist in S across batches.
__device__ void reduce_batch(const Smem &S, int NP, int max_patches, float cos_patch, float4 *scr) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int nc = S.misc[0];
    const int np0 = S.misc[1];
    // ---- Assign: join the most similar existing patch if similar enough
    for (int c = t; c < nc; c += kT) {
        V3 n = v3(S.cnx[c], S.cny[c], S.cnz[c]);
        int best = -1;
        float bd = -3.0f;
        for (int j = 0; j < np0; ++j) {
            float d = dot(n, pvec(S.pn, NP, j));
            if (d > bd) { bd = d; best = j; }
        }
        short st = -1;
        if (best >= 0 && bd >= cos_patch) {
            st = (short)best;
            V3 x = v3(S.cx[c], S.cy[c], S.cz[c]);
            V3 a = pvec(S.pa, NP, best), t1 = pvec(S.pt1, NP, best), t2 = pvec(S.pt2, NP, best);
            for (int s = 0; s < kSlots; ++s)
                atomicMax(&S.keys[s * NP + best], slot_key(slot_score(s, x, S.cphi[c], a, t1, t2), S.cidx[c]));
        }
        S.cst[c] = st;
    }
    __syncthreads();
    // slot winners of this batch publish their data
    for (int c = t; c < nc; c += kT) {
        int j = S.cst[c];
        if (j < 0) continue;
        bool won = false;
        for (int s = 0; s < kSlots; ++s) won |= (key_sample(S.keys[s * NP + j]) == S.cidx[c]);
        if (won)
            scratch_put(scr, S.cidx[c], v3(S.cx[c], S.cy[c], S.cz[c]), S.cphi[c], v3(S.cnx[c], S.cny[c], S.cnz[c]));
    }
    __syncthreads();
    // ---- while candidates remain: FindDeepest, BinReduce, AddPatch (one warp)
    if (warp == 0) {
        const int T = NP - 1;   // the patch under construction
        for (;;) {
            unsigned long long mk = kNoKey;
            for (int c = lane; c < nc; c += 32)
                if (S.cst[c] == -1) {
                    unsigned long long k = ((unsigned long long)ord_f32(S.cphi[c]) << 32) | (unsigned)c;
                    mk = (k < mk) ? k : mk;
                }
            mk = warp_min_u64(mk);
            if (mk == kNoKey) break;
            const int cb = (int)(mk & 0xFFFFFFFFull);
            V3 nb = v3(S.cnx[cb], S.cny[cb], S.cnz[cb]);
            V3 ab = v3(S.cx[cb], S.cy[cb], S.cz[cb]);
            V3 t1, t2;
            tangent_basis(nb, t1, t2);
            // BinReduce: the remaining candidates with a similar normal join
            unsigned long long lk[kSlots];
            for (int s = 0; s < kSlots; ++s) lk[s] = 0ull;
            for (int c = lane; c < nc; c += 32) {
                if (S.cst[c] != -1) continue;
                V3 n = v3(S.cnx[c], S.cny[c], S.cnz[c]);
                if (c == cb || dot(n, nb) >= cos_patch) {
                    S.cst[c] = -2;
                    V3 x = v3(S.cx[c], S.cy[c], S.cz[c]);
                    for (int s = 0; s < kSlots; ++s) {
                        unsigned long long k = slot_key(slot_score(s, x, S.cphi[c], ab, t1, t2), S.cidx[c]);
                        lk[s] = (k > lk[s]) ? k : lk[s];
                    }
                }
            }
            unsigned long long gk[kSlots];
            for (int s = 0; s < kSlots; ++s) gk[s] = warp_max_u64(lk[s]);
            // the lane holding a winner publishes its data
            for (int c = lane; c < nc; c += 32) {
                if (S.cst[c] != -2) continue;
                bool won = false;
                for (int s = 0; s < kSlots; ++s) won |= (key_sample(gk[s]) == S.cidx[c]);
                if (won)
                    scratch_put(scr, S.cidx[c], v3(S.cx[c], S.cy[c], S.cz[c]), S.cphi[c],
                                v3(S.cnx[c], S.cny[c], S.cnz[c]));
                S.cst[c] = -3;   // consumed
            }
            if (lane == 0) {
                set_pvec(S.pn, NP, T, nb); set_pvec(S.pa, NP, T, ab);
                set_pvec(S.pt1, NP, T, t1); set_pvec(S.pt2, NP, T, t2);
                for (int s = 0; s < kSlots; ++s) S.keys[s * NP + T] = gk[s];
            }
            __syncwarp();
            // AddPatch: append below capacity, else replace the most similar patch if the
            // new one measures higher, else drop it
            const int npat = S.misc[1];
            int dst = -1;
            if (npat < max_patches) {
                dst = npat;
            } else {
                unsigned long long bk = 0ull;
                for (int j = lane; j < npat; j += 32) {
                    unsigned long long k = ((unsigned long long)ord_f32(dot(nb, pvec(S.pn, NP, j))) << 32) |
                                           (unsigned)(0xFFFFFFFFu - (unsigned)j);
                    bk = (k > bk) ? k : bk;
                }
                bk = warp_max_u64(bk);
                const int ks = key_sample(bk);
                float mnew = 0.f, mold = 0.f;
                if (lane == 0) {
                    mnew = patch_measure(S, NP, T, scr);
                    mold = patch_measure(S, NP, ks, scr);
                }
                mnew = __shfl_sync(0xffffffffu, mnew, 0);
                mold = __shfl_sync(0xffffffffu, mold, 0);
                if (mnew > mold) dst = ks;
            }
            if (dst >= 0 && lane < 12) {
                float *arr = (lane < 3) ? S.pn : (lane < 6) ? S.pa : (lane < 9) ? S.pt1 : S.pt2;
                const int comp = lane % 3;
                arr[comp * NP + dst] = arr[comp * NP + T];
            }
            if (dst >= 0 && lane < kSlots) S.keys[lane * NP + dst] = S.keys[lane * NP + T];
            if (lane == 0 && dst == npat) S.misc[1] = npat + 1;
            __syncwarp();
        }
    }
    __syncthreads();
}

// Writes the reduced contacts of the pair: patches in order, distinct slot members in
// slot order.  Called by warp 0.
__device__ void emit_contacts(const Smem &S, int NP, const float4 *scr, DContact *out, int cap,
                              int *count, unsigned *status) {
    const int lane = threadIdx.x & 31;
    const int npat = S.misc[1];
    int n = 0;
    for (int j = 0; j < npat; ++j) {
        int id = -1;
        if (lane < kSlots) id = key_sample(S.keys[lane * NP + j]);
        bool dup = false;
        for (int s = 0; s < kSlots; ++s) {
            int o = __shfl_sync(0xffffffffu, id, s);
            if (s < lane && o == id) dup = true;
        }
        const bool emit = (lane < kSlots) && !dup;
        const unsigned m = __ballot_sync(0xffffffffu, emit);
        if (emit) {
            const int k = n + __popc(m & ((1u << lane) - 1u));
            if (k < cap) {
                float4 a = scr[2 * id], b = scr[2 * id + 1];
                DContact c;
                c.xa[0] = a.x; c.xa[1] = a.y; c.xa[2] = a.z; c.phi = a.w;
                c.n[0] = b.x; c.n[1] = b.y; c.n[2] = b.z;
                c.sample_patch = id | (j << 24);
                out[k] = c;
            }
        }
        n += __popc(m);
    }
    if (lane == 0) {
        if (n > cap) atomicOr(status, kStatusOverflow);
        *count = n < cap ? n : cap;
    }
}

// Appends this thread's candidate (if valid) to shared memory in (round, thread) order.
__device__ __forceinline__ void compact_push(const Smem &S, bool valid, V3 x, V3 n, float phi, int sample) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const unsigned m = __ballot_sync(0xffffffffu, valid);
    if (lane == 0) S.misc[2 + warp] = __popc(m);
    __syncthreads();
    int base = S.misc[0];
    for (int w = 0; w < warp; ++w) base += S.misc[2 + w];
    if (valid) {
        const int k = base + __popc(m & ((1u << lane) - 1u));
        S.cx[k] = x.x; S.cy[k] = x.y; S.cz[k] = x.z;
        S.cnx[k] = n.x; S.cny[k] = n.y; S.cnz[k] = n.z;
        S.cphi[k] = phi; S.cidx[k] = sample;
    }
    __syncthreads();
    if (t == 0) {
        int tot = 0;
        for (int w = 0; w < kT / 32; ++w) tot += S.misc[2 + w];
        S.misc[0] += tot;
    }
    __syncthreads();
}

__device__ __forceinline__ void init_patches(const Smem &S, int NP) {
    for (int i = threadIdx.x; i < kSlots * NP; i += kT) S.keys[i] = 0ull;
    if (threadIdx.x == 0) { S.misc[0] = 0; S.misc[1] = 0; }
}

// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kT) detect_kernel(SimParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int NP = p.max_patches + 1;
    Smem S = carve(smem_raw, NP);
    const int pi = blockIdx.x;
    const PairDev P = p.pairs[pi];
    const AssetDev ga = p.assets[P.asset_a];
    const AssetDev gb = p.assets[P.asset_b];
    __shared__ PairXf X;
    if (threadIdx.x == 0) {
        load_pose(p, P.a, X.RA, X.pA);
        load_pose(p, P.b, X.RB, X.pB);
    }
    init_patches(S, NP);
    __syncthreads();
    const PairXf Xl = X;
    float4 *scr = p.scratch + P.scratch_off;
    const float cutoff = p.contact_offset;
    for (int base = 0; base < ga.ns; base += kBatch) {
        if (threadIdx.x == 0) S.misc[0] = 0;
        __syncthreads();
        // Generate: query this batch's samples; candidates have phi < contact_offset
        for (int r = 0; r < kPerThread; ++r) {
            const int i = base + r * kT + threadIdx.x;
            V3 xw = v3(0, 0, 0), nw = v3(0, 0, 0);
            float phi = 0.f;
            bool ok = false;
            if (i < ga.ns) {
                const float4 s = __ldg(&ga.samples[i]);
                ok = query_sample(Xl, gb, s, xw, nw, phi) && (phi < cutoff);
            }
            compact_push(S, ok, xw, nw, phi, i);
        }
        reduce_batch(S, NP, p.max_patches, p.cos_patch, scr);
    }
    if (threadIdx.x < 32)
        emit_contacts(S, NP, scr, p.contacts + (long long)pi * p.cap_pair, p.cap_pair, p.counts + pi, p.status);
}

// Algorithm 1 on a candidate list in global memory (fw_candidate layout, sorted by
// sample) -- the same reduction code as detect_kernel, for parity tests.
__global__ void __launch_bounds__(kT) reduce_list_kernel(SimParams p, const float *cands, int n, float4 *scr,
                                                         DContact *out, int cap, int *count, int *npatch) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int NP = p.max_patches + 1;
    Smem S = carve(smem_raw, NP);
    init_patches(S, NP);
    __syncthreads();
    const int *ci = reinterpret_cast<const int *>(cands);
    int start = 0;
    while (start < n) {
        const int bidx = ci[8 * start] / kBatch;
        int end = start;
        while (end < n && ci[8 * end] / kBatch == bidx) ++end;
        if (threadIdx.x == 0) S.misc[0] = 0;
        __syncthreads();
        for (int c0 = start; c0 < end; c0 += kT) {
            const int c = c0 + threadIdx.x;
            const bool ok = c < end;
            V3 x = v3(0, 0, 0), nn = v3(0, 0, 0);
            float phi = 0.f;
            int sample = 0;
            if (ok) {
                const float *r = cands + 8 * c;
                sample = ci[8 * c];
                phi = r[1];
                x = v3(r[2], r[3], r[4]);
                nn = v3(r[5], r[6], r[7]);
            }
            compact_push(S, ok, x, nn, phi, sample);
        }
        reduce_batch(S, NP, p.max_patches, p.cos_patch, scr);
        start = end;
    }
    if (threadIdx.x < 32) emit_contacts(S, NP, scr, out, cap, count, p.status);
    if (threadIdx.x == 0) *npatch = S.misc[1];
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

__global__ void query_pair_kernel(SimParams p, int pi, float *phi, float *nrm) {
    const PairDev P = p.pairs[pi];
    const AssetDev ga = p.assets[P.asset_a];
    const AssetDev gb = p.assets[P.asset_b];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ga.ns) return;
    PairXf X;
    load_pose(p, P.a, X.RA, X.pA);
    load_pose(p, P.b, X.RB, X.pB);
    V3 xw, nw;
    float f;
    if (query_sample(X, gb, ga.samples[i], xw, nw, f)) {
        phi[i] = f;
        nrm[3 * i] = nw.x; nrm[3 * i + 1] = nw.y; nrm[3 * i + 2] = nw.z;
    } else {
        phi[i] = __int_as_float(0x7f800000);
        nrm[3 * i] = 0.f; nrm[3 * i + 1] = 0.f; nrm[3 * i + 2] = 0.f;
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

__global__ void __launch_bounds__(kT) reduce_noalloc_kernel(SimParams p, const float *cands, int n, float4 *scr,
                                                            fw_contact *out, int cap, int *counts) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int *ci = reinterpret_cast<const int *>(cands);
    bool bad = false;
    for (int i = threadIdx.x; i < n; i += kT) {
        const int sm = ci[8 * i];
        bad |= sm < 0 || sm >= kNoAllocMaxSamples || (i > 0 && ci[8 * (i - 1)] >= sm);
    }
    if (__syncthreads_or(bad)) {
        if (threadIdx.x == 0) { counts[0] = -1; counts[1] = 0; }
        return;
    }
    const int NP = p.max_patches + 1;
    Smem S = carve(smem_raw, NP);
    init_patches(S, NP);
    __syncthreads();
    DContact *stage = reinterpret_cast<DContact *>(scr + 2 * kNoAllocMaxSamples);
    int *stage_count = reinterpret_cast<int *>(scr + 2 * kNoAllocMaxSamples + kStageF4);
    int start = 0;
    while (start < n) {
        const int bidx = ci[8 * start] / kBatch;
        int end = start;
        while (end < n && ci[8 * end] / kBatch == bidx) ++end;
        if (threadIdx.x == 0) S.misc[0] = 0;
        __syncthreads();
        for (int c0 = start; c0 < end; c0 += kT) {
            const int c = c0 + threadIdx.x;
            const bool ok = c < end;
            V3 x = v3(0, 0, 0), nn = v3(0, 0, 0);
            float phi = 0.f;
            int sample = 0;
            if (ok) {
                const float *r = cands + 8 * c;
                sample = ci[8 * c];
                phi = r[1];
                x = v3(r[2], r[3], r[4]);
                nn = v3(r[5], r[6], r[7]);
            }
            compact_push(S, ok, x, nn, phi, sample);
        }
        reduce_batch(S, NP, p.max_patches, p.cos_patch, scr);
        start = end;
    }
    if (threadIdx.x < 32) emit_contacts(S, NP, scr, stage, p.max_patches * kSlots, stage_count, p.status);
    __syncthreads();
    const int k = *stage_count;
    for (int i = threadIdx.x; i < k && i < cap; i += kT) {
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
    if (threadIdx.x == 0) { counts[0] = k; counts[1] = S.misc[1]; }
}

}  // namespace

// The scratch of fw_reduce_noalloc: a fixed 2.2 MB block in every device that loads the
// library, shared by all calls.
static __device__ __align__(256) float4 g_noalloc[kNoAllocF4];

namespace {
float4 *g_noalloc_dev[64];    // its device address per device ordinal (0 until set up)
bool g_noalloc_ready[64];
}  // namespace

// First use on a device (that device current): look up the device address of g_noalloc
// (the host-side name is only a stand-in) and raise the kernel's shared-memory limit.
// Neither step allocates memory.
cudaError_t noalloc_setup(int device) {
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    if (g_noalloc_ready[device]) return cudaSuccess;
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(reduce_noalloc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes(kMaxPatchesCap + 1));
    if (e != cudaSuccess) return e;
    g_noalloc_dev[device] = static_cast<float4 *>(ptr);
    g_noalloc_ready[device] = true;
    return cudaSuccess;
}

cudaError_t launch_reduce_noalloc(const SimParams &p, int device, const float *d_cands, int n, fw_contact *d_out,
                                  int cap, int *d_counts, cudaStream_t s) {
    cudaError_t e = noalloc_setup(device);
    if (e != cudaSuccess) return e;
    reduce_noalloc_kernel<<<1, kT, smem_bytes(p.max_patches + 1), s>>>(p, d_cands, n, g_noalloc_dev[device], d_out,
                                                                        cap, d_counts);
    return cudaGetLastError();
}

size_t detect_smem_bytes(int max_patches) { return smem_bytes(max_patches + 1); }

// Raises the kernels' dynamic shared-memory limit (outside any stream capture).
cudaError_t prepare_detect(int max_patches) {
    const int sm = (int)smem_bytes(max_patches + 1);
    cudaError_t e = cudaFuncSetAttribute(detect_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(reduce_list_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

cudaError_t launch_detect(const SimParams &p, cudaStream_t s) {
    if (p.n_pairs == 0) return cudaSuccess;
    detect_kernel<<<p.n_pairs, kT, smem_bytes(p.max_patches + 1), s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_reduce_list(const SimParams &p, const float *d_cands, int n, DContact *out, int *d_count,
                               int *d_npatch, cudaStream_t s) {
    reduce_list_kernel<<<1, kT, smem_bytes(p.max_patches + 1), s>>>(p, d_cands, n, p.scratch, out,
                                                                     p.max_patches * kSlots, d_count, d_npatch);
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
