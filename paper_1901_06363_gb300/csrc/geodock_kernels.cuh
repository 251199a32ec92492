// Device code of the batched pose evaluator (GeoDock-MA, Alg. 1/2, Eq. 1).
//
// Work decomposition. A warp owns G = 32/Q initial poses of ONE ligand in ONE
// pocket; Q lanes share a pose and split its candidate angles. Because every
// pose of a warp has the same topology, loops over atoms, fragments and
// angles are warp-uniform; only coordinates differ per lane. Coordinates of
// the warp's poses live in shared memory as [atom][axis][pose] in grid units
// of the pocket, shifted so that floor(t) is the nearest voxel.
//
// Per fragment sweep (Alg. 1), with c the fragment's bond atom (on the axis)
// and k the unit bond axis, every moving atom x is split once into
//   a = c + k (k.(x-c)),  u = (x-c) - k (k.(x-c)),  w = k x u,
// so the candidate at angle theta is a + cos(theta) u + sin(theta) w (Rodrigues'
// formula). A lane keeps a chunk of KC angles' partial scores in registers
// and walks the moving atoms once per chunk. The fixed atoms' part of the
// score is summed once per sweep.
//
// Score (Eq. 1): o = l / (h^2 S), S = sum_i K(voxel(x_i)) in grid units with K
// the floored integer field, so S is an exact integer (nearest mode) and the
// argmax is an exact integer comparison. Trilinear mode interpolates K.
//
// Bump check (Alg. 1 "the ligand shape is feasible"): pairs (i in M\{c},
// j in F\{b}). For atom i on its circle (centre a, radius r = |u|) and a fixed
// atom y, |x(theta) - y| >= |a - y| - r, so a pair with |a - y| >= thr + r +
// margin can never clash and is skipped; the rest are tested per angle with
// d^2(theta) = |a-y|^2 + r^2 + cos(theta) 2(a-y).u + sin(theta) 2(a-y).w.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gd {

constexpr unsigned FULL = 0xffffffffu;

struct PocketDev {
    const uint16_t* K;  // floored field, x fastest
    int nx, ny, nz;
    double h;  // voxel edge (Å)
    double origin[3];
    double centre[3];
};

struct LigDev {
    int atom_off;  // first atom in the batch arrays
    int l;         // atoms
    int nside;     // 2 * rotatable bonds
    int side_off;  // first fragment-sweep descriptor
    double g[3];   // centroid of the input conformer (Å)
    int64_t id;    // seeds the initial orientations
};

// One fragment sweep. Atom-index pool layout per sweep: the moving atoms
// M\{c} (nmov of them), then F\{b} (nfixB), then b, then c; so F\{b} is the
// bump partner list and F\{b} + b + c (nfixS = nfixB + 2) the fixed part of
// the score.
struct SideDev {
    int mov_off, fix_off;
    uint8_t c, b, m, nmov, nfixB, nfixS, pad0, pad1;
};

struct TraceDev {
    int pmax;
    int32_t* chosen_k;
    float* cand_S;
    int32_t* cand_status;
    float* pose_S;
    float* pose_init_S;
    int32_t* pose_status;
    float* init_xyz;
    float* pose_xyz;
};

struct SweepParams {
    const LigDev* lig;
    const SideDev* side;
    const uint8_t* idx;
    const float* xyz0;  // input coordinates, 3 per atom (Å)
    const PocketDev* pockets;
    const int2* tasks;  // (pair, pose group); pair = pocket * nlig + ligand
    int ntask;
    int nlig;
    int natoms;          // atoms in the batch
    unsigned* counter;   // work queue head (scratch, zeroed before launch)
    int n_poses;
    int repetitions;
    int Q;               // lanes per pose
    int lmax;            // largest ligand of the batch (shared-memory stride)
    double threshold;
    double bump_thr;     // Å
    uint64_t seed;
    const float2* cs_hp;  // cos/sin of k * hp_step, k = 0..P_hp-1
    const float2* cs_lp;
    int P_hp, P_lp;
    // tile peeling
    int peel;            // 1: hp sweeps use tile peeling
    const float2* cs_peel;  // cos/sin of the tile centres
    int n_tiles;         // 360 / tile
    int per_tile;        // tile / hp_step
    // per-pose results (scratch)
    unsigned long long* pose_key;  // (float bits of S) << 32 | pose; ~0 when skipped
    float* pose_xyz;               // grid units, ((pocket*natoms + atom_off)*N + p*l + i)*3
    int trace_on;
    TraceDev tr;
};

// ------------------------------------------------------------------ helpers

// floor(t) as an unsigned voxel index, for 0 <= t < 2^23: adding 2^23 with
// round-toward-zero leaves floor(t) in the low mantissa bits. Any t < 0 (or
// NaN) yields an index >= 2^31, i.e. outside every grid.
__device__ __forceinline__ uint32_t vox(float t) {
    return __float_as_uint(__fadd_rz(t, 8388608.0f)) - 0x4B000000u;
}

__device__ __forceinline__ float3 ld3(const float* xs, int i, int G, int ps) {
    return make_float3(xs[(3 * i) * G + ps], xs[(3 * i + 1) * G + ps], xs[(3 * i + 2) * G + ps]);
}
__device__ __forceinline__ void st3(float* xs, int i, int G, int ps, float3 v) {
    xs[(3 * i) * G + ps] = v.x;
    xs[(3 * i + 1) * G + ps] = v.y;
    xs[(3 * i + 2) * G + ps] = v.z;
}

// Rodrigues split of x about the axis through c along unit k (explicit
// roundings so the commit reproduces the candidate bit for bit).
struct Split {
    float3 a, u, w;
};
__device__ __forceinline__ Split split(float3 x, float3 c, float3 k) {
    float vx = __fsub_rn(x.x, c.x), vy = __fsub_rn(x.y, c.y), vz = __fsub_rn(x.z, c.z);
    float kv = __fmaf_rn(k.z, vz, __fmaf_rn(k.y, vy, __fmul_rn(k.x, vx)));
    Split s;
    s.a = make_float3(__fmaf_rn(k.x, kv, c.x), __fmaf_rn(k.y, kv, c.y), __fmaf_rn(k.z, kv, c.z));
    s.u = make_float3(__fmaf_rn(-k.x, kv, vx), __fmaf_rn(-k.y, kv, vy), __fmaf_rn(-k.z, kv, vz));
    s.w = make_float3(__fmaf_rn(k.y, s.u.z, -__fmul_rn(k.z, s.u.y)), __fmaf_rn(k.z, s.u.x, -__fmul_rn(k.x, s.u.z)),
                      __fmaf_rn(k.x, s.u.y, -__fmul_rn(k.y, s.u.x)));
    return s;
}
__device__ __forceinline__ float3 place(const Split& s, float cs, float sn) {
    return make_float3(__fmaf_rn(sn, s.w.x, __fmaf_rn(cs, s.u.x, s.a.x)),
                       __fmaf_rn(sn, s.w.y, __fmaf_rn(cs, s.u.y, s.a.y)),
                       __fmaf_rn(sn, s.w.z, __fmaf_rn(cs, s.u.z, s.a.z)));
}

// Field term of one atom at shifted grid position t.
// MODE 0 nearest (t shifted by +0.5: voxel = floor(t), inside iff 0 <= t < n)
// MODE 1 trilinear (unshifted: inside iff 0 <= t <= n-1)
// Returns the term; *in reports whether the atom is inside the box. With
// CLIP the value is only meaningful when inside; without CLIP the lookup is
// clamped and the squared excess outside the box is added.
template <int MODE, bool CLIP>
__device__ __forceinline__ float term(const PocketDev& pd, const uint16_t* __restrict__ K, float3 t, bool* in) {
    if (MODE == 0) {
        uint32_t ix = vox(t.x), iy = vox(t.y), iz = vox(t.z);
        bool inside = (ix < (uint32_t)pd.nx) & (iy < (uint32_t)pd.ny) & (iz < (uint32_t)pd.nz);
        *in = inside;
        if (CLIP) {
            uint32_t id = inside ? ix + (uint32_t)pd.nx * (iy + (uint32_t)pd.ny * iz) : 0u;
            return (float)__ldg(K + id);
        } else {
            int cx = min(max((int)ix, 0), pd.nx - 1), cy = min(max((int)iy, 0), pd.ny - 1),
                cz = min(max((int)iz, 0), pd.nz - 1);
            float v = (float)__ldg(K + (cx + pd.nx * (cy + pd.ny * cz)));
            float ex = fmaxf(-t.x, 0.f) + fmaxf(t.x - (float)pd.nx, 0.f);
            float ey = fmaxf(-t.y, 0.f) + fmaxf(t.y - (float)pd.ny, 0.f);
            float ez = fmaxf(-t.z, 0.f) + fmaxf(t.z - (float)pd.nz, 0.f);
            return inside ? v : v + (ex * ex + ey * ey + ez * ez);
        }
    } else {
        float hx = (float)(pd.nx - 1), hy = (float)(pd.ny - 1), hz = (float)(pd.nz - 1);
        bool inside = (t.x >= 0.f) & (t.x <= hx) & (t.y >= 0.f) & (t.y <= hy) & (t.z >= 0.f) & (t.z <= hz);
        *in = inside;
        float cx = fminf(fmaxf(t.x, 0.f), hx), cy = fminf(fmaxf(t.y, 0.f), hy), cz = fminf(fmaxf(t.z, 0.f), hz);
        int ix = min((int)vox(cx), pd.nx - 2), iy = min((int)vox(cy), pd.ny - 2), iz = min((int)vox(cz), pd.nz - 2);
        float fx = cx - (float)ix, fy = cy - (float)iy, fz = cz - (float)iz;
        const uint16_t* p = K + (ix + pd.nx * (iy + pd.ny * iz));
        int sy = pd.nx, sz = pd.nx * pd.ny;
        float c000 = __ldg(p), c100 = __ldg(p + 1), c010 = __ldg(p + sy), c110 = __ldg(p + sy + 1);
        float c001 = __ldg(p + sz), c101 = __ldg(p + sz + 1), c011 = __ldg(p + sz + sy), c111 = __ldg(p + sz + sy + 1);
        float c00 = fmaf(fx, c100 - c000, c000), c10 = fmaf(fx, c110 - c010, c010);
        float c01 = fmaf(fx, c101 - c001, c001), c11 = fmaf(fx, c111 - c011, c011);
        float c0 = fmaf(fy, c10 - c00, c00), c1 = fmaf(fy, c11 - c01, c01);
        float v = fmaf(fz, c1 - c0, c0);
        if (CLIP) return v;
        float ex = t.x - cx, ey = t.y - cy, ez = t.z - cz;
        return v + (ex * ex + ey * ey + ez * ez);
    }
}

// --------------------------------------------------------- initial poses

__device__ __forceinline__ uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}
// Output number ctr+1 of SplitMix64 seeded with `seed`, in [0, 1).
__device__ __forceinline__ double unif(uint64_t seed, uint64_t ctr) {
    return (double)(sm_mix(seed + (ctr + 1) * 0x9e3779b97f4a7c15ULL) >> 11) * 0x1.0p-53;
}
// Identity for pose 0; otherwise a uniform random rotation from Shoemake's
// quaternion construction (three uniforms per pose, counter-based).
__device__ __forceinline__ void pose_matrix(uint64_t seed, int64_t id, int p, double* R) {
    if (p == 0) {
        R[0] = 1; R[1] = 0; R[2] = 0; R[3] = 0; R[4] = 1; R[5] = 0; R[6] = 0; R[7] = 0; R[8] = 1;
        return;
    }
    uint64_t base = ((uint64_t)id * 4096ull + (uint64_t)p) * 4ull;
    double u1 = unif(seed, base), u2 = unif(seed, base + 1), u3 = unif(seed, base + 2);
    double r1 = sqrt(1.0 - u1), r2 = sqrt(u1);
    double s2, c2, s3, c3;
    sincospi(2.0 * u2, &s2, &c2);
    sincospi(2.0 * u3, &s3, &c3);
    double x = r1 * s2, y = r1 * c2, z = r2 * s3, w = r2 * c3;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - z * w); R[2] = 2 * (x * z + y * w);
    R[3] = 2 * (x * y + z * w); R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - x * w);
    R[6] = 2 * (x * z - y * w); R[7] = 2 * (y * z + x * w); R[8] = 1 - 2 * (x * x + y * y);
}

// Minimum of 64-bit keys over the Q lanes that share a pose.
__device__ __forceinline__ unsigned long long group_min(unsigned long long v, int Q) {
    for (int off = Q >> 1; off > 0; off >>= 1) {
        unsigned long long o = __shfl_xor_sync(FULL, v, off);
        v = o < v ? o : v;
    }
    return v;
}
__device__ __forceinline__ float group_sum(float v, int Q) {
    for (int off = Q >> 1; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
    return v;
}
__device__ __forceinline__ bool group_all(bool v, int Q) {
    int x = v ? 1 : 0;
    for (int off = Q >> 1; off > 0; off >>= 1) x &= __shfl_xor_sync(FULL, x, off);
    return x != 0;
}

__device__ __forceinline__ unsigned long long make_key(float S, int k) {
    return ((unsigned long long)__float_as_uint(S) << 32) | (unsigned)k;
}

// ------------------------------------------------------------- sweep kernel

// One pass over a chunk of up to KC candidate angles of one fragment sweep,
// for the lane's pose. Returns the best (S, slot) key among the chunk's
// feasible candidates, or ~0.
template <int KC, int MODE, bool CLIP>
__device__ __forceinline__ unsigned long long sweep_chunk(const PocketDev& pd, const uint16_t* __restrict__ K,
                                                          const float* xs, int G, int ps,
                                                          const uint8_t* __restrict__ mov, int nmov,
                                                          const uint8_t* __restrict__ fixB, int nfixB, float3 gc,
                                                          float3 kax, float thr_g, float S_fix, bool live,
                                                          const float2 (&csj)[KC], int slot_start, int slot_step,
                                                          int nvalid, float* trace_S, int* trace_st) {
    float cj[KC], sj[KC];
#pragma unroll
    for (int j = 0; j < KC; ++j) {
        cj[j] = csj[j].x;
        sj[j] = csj[j].y;
    }
    float acc[KC];
#pragma unroll
    for (int j = 0; j < KC; ++j) acc[j] = 0.f;
    unsigned long long bad = 0ull, box = 0ull;
    const float thr2 = thr_g * thr_g;

    for (int im = 0; im < nmov; ++im) {
        const int i = mov[im];
        Split s = split(ld3(xs, i, G, ps), gc, kax);
#pragma unroll
        for (int j = 0; j < KC; ++j) {
            bool in;
            acc[j] += term<MODE, CLIP>(pd, K, place(s, cj[j], sj[j]), &in);
            if (CLIP && !in) box |= 1ull << j;
        }
        // bump pairs of this moving atom
        float r2 = s.u.x * s.u.x + s.u.y * s.u.y + s.u.z * s.u.z;
        float R = thr_g + sqrtf(r2) + 1e-3f;
        float R2 = R * R;
        for (int f = 0; f < nfixB; ++f) {
            float3 y = ld3(xs, fixB[f], G, ps);
            float dx = s.a.x - y.x, dy = s.a.y - y.y, dz = s.a.z - y.z;
            float dd = dx * dx + dy * dy + dz * dz;
            bool risk = live && dd < R2;
            if (__any_sync(FULL, risk)) {
                if (risk) {
                    float A = dd + r2 - thr2;
                    float B = 2.f * (dx * s.u.x + dy * s.u.y + dz * s.u.z);
                    float C = 2.f * (dx * s.w.x + dy * s.w.y + dz * s.w.z);
#pragma unroll
                    for (int j = 0; j < KC; ++j)
                        if (fmaf(sj[j], C, fmaf(cj[j], B, A)) < 0.f) bad |= 1ull << j;
                }
            }
        }
    }
    unsigned long long best = ~0ull;
#pragma unroll
    for (int j = 0; j < KC; ++j) {
        if (j < nvalid) {
            float S = S_fix + acc[j];
            bool clash = (bad >> j) & 1ull, out = (box >> j) & 1ull;
            const int slot = slot_start + slot_step * j;
            if (trace_S) {
                trace_S[slot] = S;
                trace_st[slot] = clash ? 0 : (out ? -1 : 1);
            }
            if (!clash && !out) {
                unsigned long long key = make_key(S, slot);
                best = key < best ? key : best;
            }
        }
    }
    return best;
}

template <int KC, int MODE, bool CLIP>
__global__ void __launch_bounds__(256) sweep_kernel(SweepParams P) {
    extern __shared__ float smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int Q = P.Q;
    const int G = 32 / Q;
    const int ps = lane / Q;
    const int q = lane % Q;
    float* xs = smem + (size_t)warp * P.lmax * 3 * G;
    const float shift = MODE == 0 ? 0.5f : 0.0f;

    for (;;) {
        int task = 0;
        if (lane == 0) task = (int)atomicAdd(P.counter, 1u);
        task = __shfl_sync(FULL, task, 0);
        if (task >= P.ntask) break;
        const int2 tk = P.tasks[task];
        const int pocket = tk.x / P.nlig, b = tk.x % P.nlig;
        const PocketDev& pd = P.pockets[pocket];
        const uint16_t* __restrict__ K = pd.K;
        const LigDev L = P.lig[b];
        const int p = tk.y * G + ps;
        const bool active = p < P.n_poses;
        const float thr_g = (float)(P.bump_thr / pd.h);

        // ---- initial rigid orientation (FP64), centroid on the pocket centre
        {
            double R[9];
            pose_matrix(P.seed, L.id, active ? p : 0, R);
            for (int i = q; i < L.l; i += Q) {
                const float* x0 = P.xyz0 + 3 * (L.atom_off + i);
                double d0 = (double)x0[0] - L.g[0], d1 = (double)x0[1] - L.g[1], d2 = (double)x0[2] - L.g[2];
                float3 t;
                t.x = (float)((pd.centre[0] + (R[0] * d0 + R[1] * d1 + R[2] * d2) - pd.origin[0]) / pd.h + shift);
                t.y = (float)((pd.centre[1] + (R[3] * d0 + R[4] * d1 + R[5] * d2) - pd.origin[1]) / pd.h + shift);
                t.z = (float)((pd.centre[2] + (R[6] * d0 + R[7] * d1 + R[8] * d2) - pd.origin[2]) / pd.h + shift);
                st3(xs, i, G, ps, t);
            }
        }
        __syncwarp();
        float S_inc = 0.f;
        bool inbox = true;
        {
            const int i0 = MODE == 0 ? q : 0, di = MODE == 0 ? Q : 1;
            for (int i = i0; i < L.l; i += di) {
                bool in;
                S_inc += term<MODE, CLIP>(pd, K, ld3(xs, i, G, ps), &in);
                inbox = inbox && in;
            }
            if (MODE == 0) {
                S_inc = group_sum(S_inc, Q);
                inbox = group_all(inbox, Q);
            }
        }
        const bool live = active && (!CLIP || inbox);
        const int nsweep = P.repetitions * L.nside;
        // trace layout: n_poses * repetitions * (sweeps of earlier ligands) + p * nsweep
        const int64_t tbase = (int64_t)P.n_poses * P.repetitions * L.side_off + (int64_t)p * nsweep;
        if (P.trace_on && active && q == 0) {
            int64_t pi = (int64_t)b * P.n_poses + p;
            P.tr.pose_init_S[pi] = S_inc;
            P.tr.pose_status[pi] = live ? 0 : 1;
            for (int i = 0; i < L.l; ++i) {
                float3 t = ld3(xs, i, G, ps);
                float* o = P.tr.init_xyz + ((int64_t)L.atom_off * P.n_poses + (int64_t)p * L.l + i) * 3;
                o[0] = (float)(((double)t.x - shift) * pd.h + pd.origin[0]);
                o[1] = (float)(((double)t.y - shift) * pd.h + pd.origin[1]);
                o[2] = (float)(((double)t.z - shift) * pd.h + pd.origin[2]);
            }
        }

        if (__any_sync(FULL, live)) {
            for (int rep = 0; rep < P.repetitions; ++rep) {
                for (int si = 0; si < L.nside; ++si) {
                    const SideDev sd = P.side[L.side_off + si];
                    const int sweep = rep * L.nside + si;
                    const bool coarse = (double)sd.m / (double)L.l <= P.threshold;
                    const bool peel = P.peel && !coarse;
                    float* tS = nullptr;
                    int* tSt = nullptr;
                    if (P.trace_on && active) {
                        int64_t ci = (tbase + sweep) * P.tr.pmax;
                        tS = P.tr.cand_S + ci;
                        tSt = P.tr.cand_status + ci;
                        for (int j = q; j < P.tr.pmax; j += Q) {
                            tS[j] = 0.f;
                            tSt[j] = -2;
                        }
                        if (q == 0) {
                            tS[0] = S_inc;
                            tSt[0] = 1;
                        }
                    }
                    __syncwarp();
                    const float3 gc = ld3(xs, sd.c, G, ps), gb = ld3(xs, sd.b, G, ps);
                    float3 kax = make_float3(gc.x - gb.x, gc.y - gb.y, gc.z - gb.z);
                    {
                        float inv = rsqrtf(kax.x * kax.x + kax.y * kax.y + kax.z * kax.z);
                        kax.x *= inv;
                        kax.y *= inv;
                        kax.z *= inv;
                    }
                    // fixed atoms' part of S (F plus the axis atom c). Nearest-mode terms
                    // are integers, so splitting them over the pose's lanes is exact;
                    // trilinear sums stay in one fixed order for every tile shape.
                    float S_fix = 0.f;
                    const uint8_t* fixS = P.idx + sd.fix_off;
                    {
                        const int i0 = MODE == 0 ? q : 0, di = MODE == 0 ? Q : 1;
                        for (int i = i0; i < sd.nfixS; i += di) {
                            bool in;
                            S_fix += term<MODE, CLIP>(pd, K, ld3(xs, fixS[i], G, ps), &in);
                        }
                        if (MODE == 0) S_fix = group_sum(S_fix, Q);
                    }
                    const uint8_t* mov = P.idx + sd.mov_off;
                    const uint8_t* fixB = P.idx + sd.fix_off;

                    unsigned long long best = make_key(S_inc, 0);
                    const float2* cs = coarse ? P.cs_lp : P.cs_hp;
                    // candidate phases: flat sweep, or tile centres then the best tile
                    int phases = peel ? 2 : 1;
                    int tile_first = 0;  // first angle index of the best tile (hp table)
                    bool have_tile = true;  // a pose with no feasible tile centre keeps its incumbent
                    for (int ph = 0; ph < phases; ++ph) {
                        int ncand, slot0;
                        const float2* tab;
                        if (!peel) {
                            ncand = (coarse ? P.P_lp : P.P_hp) - 1;
                            tab = cs + 1;
                            slot0 = 1;
                        } else if (ph == 0) {
                            ncand = P.n_tiles;
                            tab = P.cs_peel;
                            slot0 = 1;
                        } else {
                            ncand = P.per_tile;
                            tab = P.cs_hp + tile_first;
                            slot0 = 1 + P.n_tiles;
                        }
                        unsigned long long pbest = ~0ull;
                        // lane q takes candidates q, q+Q, q+2Q, ...
                        const int per_lane = (ncand + Q - 1) / Q;
                        for (int j0 = 0; j0 < per_lane; j0 += KC) {
                            float2 csj[KC];
                            int nvalid = 0;
#pragma unroll
                            for (int j = 0; j < KC; ++j) {
                                int c = q + Q * (j0 + j);
                                bool ok = (j0 + j) < per_lane && c < ncand && have_tile;
                                const float2 v = tab[ok ? c : 0];  // index 0 is always in the table
                                csj[j] = ok ? v : make_float2(1.f, 0.f);
                                nvalid += ok ? 1 : 0;
                            }
                            // valid candidates of a lane are a prefix of its chunk
                            unsigned long long cb = sweep_chunk<KC, MODE, CLIP>(
                                pd, K, xs, G, ps, mov, sd.nmov, fixB, sd.nfixB, gc, kax, thr_g, S_fix,
                                live && have_tile, csj, slot0 + q + Q * j0, Q, nvalid, tS, tSt);
                            pbest = cb < pbest ? cb : pbest;
                        }
                        pbest = group_min(pbest, Q);
                        if (peel && ph == 0) {
                            // the best tile centre picks the tile; the tile's angles are the next phase
                            have_tile = pbest != ~0ull;
                            int t = have_tile ? (int)(pbest & 0xffffffffu) - 1 : 0;
                            tile_first = t * P.per_tile;
                        } else {
                            best = pbest < best ? pbest : best;
                        }
                    }
                    best = group_min(best, Q);
                    const int kb = (int)(best & 0xffffffffu);
                    if (live && kb != 0) {
                        float2 v;
                        if (!peel) v = cs[kb];
                        else v = P.cs_hp[tile_first + (kb - 1 - P.n_tiles)];
                        if (q == 0) {
                            for (int im = 0; im < sd.nmov; ++im) {
                                const int i = mov[im];
                                Split s = split(ld3(xs, i, G, ps), gc, kax);
                                st3(xs, i, G, ps, place(s, v.x, v.y));
                            }
                        }
                        S_inc = __uint_as_float((unsigned)(best >> 32));
                    }
                    if (P.trace_on && active && q == 0) P.tr.chosen_k[tbase + sweep] = live ? kb : 0;
                    __syncwarp();
                }
            }
        }
        // ---- per-pose result
        if (active && q == 0) {
            int64_t pi = (int64_t)tk.x * P.n_poses + p;
            P.pose_key[pi] = live ? make_key(S_inc, p) : ~0ull;
            float* o = P.pose_xyz + ((int64_t)pocket * P.natoms * P.n_poses + (int64_t)L.atom_off * P.n_poses +
                                     (int64_t)p * L.l) * 3;
            for (int i = 0; i < L.l; ++i) {
                float3 t = ld3(xs, i, G, ps);
                o[3 * i] = t.x;
                o[3 * i + 1] = t.y;
                o[3 * i + 2] = t.z;
            }
            if (P.trace_on) {
                int64_t ti = (int64_t)b * P.n_poses + p;
                P.tr.pose_S[ti] = live ? S_inc : 0.f;
                for (int i = 0; i < L.l; ++i) {
                    float3 t = ld3(xs, i, G, ps);
                    float* w = P.tr.pose_xyz + ((int64_t)L.atom_off * P.n_poses + (int64_t)p * L.l + i) * 3;
                    w[0] = (float)(((double)t.x - shift) * pd.h + pd.origin[0]);
                    w[1] = (float)(((double)t.y - shift) * pd.h + pd.origin[1]);
                    w[2] = (float)(((double)t.z - shift) * pd.h + pd.origin[2]);
                }
            }
        }
        __syncwarp();
    }
}

struct FinalParams {
    int pair0;          // first (pocket, ligand) pair of this launch
    const LigDev* lig;
    const PocketDev* pockets;
    const unsigned long long* pose_key;
    const float* pose_xyz;
    int npairs, nlig, natoms, n_poses;
    float shift;
    float* score;       // dock_result array as raw words (score, pose, status, reserved)
    float* xyz_out;     // nullable, Å, ((pocket*natoms + atom_off) + i)*3
};

#ifdef GD_DEFINE_AUX_KERNELS
// ---------------------------------------------------------- finalize kernel



// One warp per (pocket, ligand): best pose over the initial poses (lowest S,
// ties to the lowest pose), its coordinates back to Å.
__global__ void finalize_kernel(FinalParams F) {
    const int lane = threadIdx.x & 31;
    const int pair = F.pair0 + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (pair >= F.pair0 + F.npairs) return;
    const int pocket = pair / F.nlig, b = pair % F.nlig;
    const LigDev L = F.lig[b];
    const PocketDev& pd = F.pockets[pocket];
    unsigned long long best = ~0ull;
    for (int p = lane; p < F.n_poses; p += 32) {
        unsigned long long k = F.pose_key[(int64_t)pair * F.n_poses + p];
        best = k < best ? k : best;
    }
    for (int off = 16; off > 0; off >>= 1) {
        unsigned long long o = __shfl_xor_sync(FULL, best, off);
        best = o < best ? o : best;
    }
    const bool ok = best != ~0ull;
    const int p = ok ? (int)(best & 0xffffffffu) : -1;
    if (lane == 0) {
        float S = __uint_as_float((unsigned)(best >> 32));
        int32_t* w = reinterpret_cast<int32_t*>(F.score + (int64_t)pair * 4);
        F.score[(int64_t)pair * 4] = ok ? (float)((double)L.l / (pd.h * pd.h * (double)S)) : 0.f;
        w[1] = p;
        w[2] = ok ? 0 : 1;
        w[3] = 0;
    }
    if (F.xyz_out) {
        const int pp = ok ? p : 0;
        const float* src = F.pose_xyz + ((int64_t)pocket * F.natoms * F.n_poses + (int64_t)L.atom_off * F.n_poses +
                                         (int64_t)pp * L.l) * 3;
        float* dst = F.xyz_out + ((int64_t)pocket * F.natoms + L.atom_off) * 3;
        for (int e = lane; e < 3 * L.l; e += 32) {
            int a = e % 3;
            dst[e] = (float)(((double)src[e] - F.shift) * pd.h + pd.origin[a]);
        }
    }
}

// ------------------------------------------------------------ field kernel

// K(v) = max(min_j |v - p_j|^2, 1), exact integers; one thread per voxel,
// probe points staged through shared memory.
__global__ void field_kernel(uint16_t* K, int nx, int ny, int nz, const int4* pts, int npts) {
    __shared__ int4 sp[256];
    const int64_t nvox = (int64_t)nx * ny * nz;
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int x = 0, y = 0, z = 0;
    if (v < nvox) {
        x = (int)(v % nx);
        y = (int)((v / nx) % ny);
        z = (int)(v / ((int64_t)nx * ny));
    }
    int best = 0x7fffffff;
    for (int base = 0; base < npts; base += 256) {
        __syncthreads();
        if (base + (int)threadIdx.x < npts) sp[threadIdx.x] = pts[base + threadIdx.x];
        __syncthreads();
        int n = min(256, npts - base);
        for (int j = 0; j < n; ++j) {
            int dx = x - sp[j].x, dy = y - sp[j].y, dz = z - sp[j].z;
            best = min(best, dx * dx + dy * dy + dz * dz);
        }
    }
    if (v < nvox) K[v] = (uint16_t)max(best, 1);
}
#endif  // GD_DEFINE_AUX_KERNELS

}  // namespace gd
