// Device code of the batched pose evaluator (GeoDock-MA, Alg. 1/2, Eq. 1).
//
// Work decomposition. A warp owns G = 32/Q initial poses of ONE ligand in ONE
// pocket; the Q lanes of a pose split its moving atoms (and its fixed atoms
// for the fixed part of the score). Because every pose of a warp has the same
// topology, loops over atoms, fragments and angles are warp-uniform; only
// coordinates differ per lane. Coordinates of the warp's poses live in shared
// memory as [atom][axis][pose] in grid units of the pocket, shifted so that
// floor(t) is the nearest voxel.
//
// Per fragment sweep (Alg. 1), with c the fragment's bond atom (on the axis)
// and k the unit bond axis, every moving atom x is split into
//   a = c + k (k.(x-c)),  u = (x-c) - k (k.(x-c)),  w = k x u,
// so the candidate at angle theta is a + cos(theta) u + sin(theta) w (Rodrigues'
// formula). A lane keeps a chunk of KC angles' partial scores in registers
// and walks its moving atoms once per chunk; the pose's lanes then add their
// partial sums. The fixed atoms' part of the score is summed once per sweep.
//
// Score (Eq. 1): o = l / (h^2 S), S = sum_i K(voxel(x_i)) in grid units with K
// the floored integer field, so S is an exact integer (nearest mode) and the
// argmax is an exact integer comparison. Trilinear mode interpolates K; the
// exact mode takes Eq. 1's inner minimum over the pocket points directly.
//
// Bump check (Alg. 1's feasibility test of the shape): pairs (i in M\{c},
// j in F\{b}). Atom i moves on a circle of radius r about the axis at axial
// position h; a fixed atom y at radius rho and axial position t comes no
// closer than sqrt((rho - r)^2 + (t - h)^2), so a pair whose closest approach
// exceeds the threshold (plus a margin for FP32 rounding) is skipped; the rest
// are tested at every candidate with
// d^2(theta) = |a-y|^2 + r^2 + cos(theta) 2(a-y).u + sin(theta) 2(a-y).w.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gd {

constexpr unsigned FULL = 0xffffffffu;

// Margin (voxels) of the padded copy of the field: cells outside the grid
// hold OUTSIDE, so a sum over atoms is >= OUTSIDE exactly when one of them
// lies outside the box (255 atoms x 2^24 < 2^32, and sums of in-box values
// stay below 255 x 65535 < 2^24).
constexpr int PAD = 16;
constexpr uint32_t OUTSIDE = 1u << 24;

struct PocketDev {
    const uint16_t* K;   // floored field, x fastest
    unsigned long long Kt;  // the same values padded by PAD voxels per side, OUTSIDE beyond the grid, as
                            // a 3D texture (point sampling, unnormalized coordinates): a fetch at padded
                            // position t returns the value of the voxel floor(t)
    unsigned long long Kc;  // the 2x2x2 corners of every voxel (i..i+1 per axis, repeated at the upper edges),
                            // eight 16-bit values per texel, as a 3D texture: one fetch per trilinear term
    const float4* pts;   // probe points (voxel index + 0.5, grid units) for the exact score; NULL if unknown
    int npts;
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
    const int2* tasks;  // (pair, group | log2(lanes per pose) << 16); pair = pocket * nlig + ligand
    int ntask;
    int slice;           // floats of shared memory per warp for its poses' coordinates
    int bw;              // 64-bit bump words per lane (ceil of the largest phase / 64)
    int nlig;
    int natoms;          // atoms in the batch
    unsigned* counter;   // work queue head (scratch, zeroed before launch)
    int n_poses;
    int repetitions;
    double threshold;
    const uint8_t* coarse;  // per sweep descriptor: 1 when its relative size m/l <= threshold (Alg. 2),
                            // decided on the host; NULL: decided here (an FP64 division per sweep)
    double bump_thr;     // Å
    uint64_t seed;
    const float2* cs_hp;  // cos/sin of k * hp_step, k = 0..P_hp-1
    const float2* cs_lp;
    int P_hp, P_lp;
    // tile peeling
    float hp_step, lp_step, tile;  // degrees
    int peel;            // 1: hp sweeps use tile peeling
    const float2* cs_peel;  // cos/sin of the tile centres
    int n_tiles;         // 360 / tile
    int per_tile;        // tile / hp_step
    // per-pose results (scratch)
    unsigned long long* pose_key;  // (float bits of S) << 32 | pose; ~0 when skipped
    unsigned* skipped;             // per pair: pose-repetitions left out at a fixed point (nullable)
    unsigned long long* lookups_skipped;  // (pose, candidate, moving atom) lookups left out because every
                                          // working pose of the warp had the candidates' block infeasible
                                          // (nullable)
    float* pose_xyz;               // grid units, ((pocket*natoms + atom_off)*N + p*l + i)*3
    int trace_on;
    TraceDev tr;
    // kept at the end: placed after `ntask` these fields cost the sweep about 3 % (measured)
    int npockets;        // pockets of the run (pair = pocket * nlig + ligand)
    int nidx;            // bytes of the batch's atom-index pool
    unsigned long long* check;  // checked builds: the first failed index check, (code << 32) | index
};

// ------------------------------------------------------------------ helpers

// Checked builds (GEODOCK_CHECKED): an index that a kernel derives from its
// inputs is tested before use; a failed test records (code << 32) | index in
// the run's status word (the first failure wins) and the access is skipped,
// so the host can report the bad index instead of the GPU faulting. Codes:
// 1 ligand atoms beyond the batch, 2 a pose group larger than its coordinate
// slice, 3 index lists beyond the pool or the staging area, 4 an atom index
// beyond its ligand, 5 a phase with more candidates than bump words, 6 a
// per-pose output beyond the run, 7 a pocket beyond the run, 8 a torsion or
// bump-pair row beyond the batch (refinement). Other builds test nothing.
#ifdef GEODOCK_CHECKED
__device__ __forceinline__ bool check_ok(unsigned long long* st, bool cond, unsigned code, unsigned long long idx) {
    if (!cond && st) atomicCAS(st, 0ull, ((unsigned long long)code << 32) | (idx & 0xffffffffull));
    return cond;
}
#define GD_OK(st, cond, code, idx) ::gd::check_ok((st), (cond), (code), (unsigned long long)(idx))
#else
#define GD_OK(st, cond, code, idx) true
#endif

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
// The same circle with its angle origin turned by r = (cos, sin): the
// candidate at angle phi of the result is the one at angle (origin + phi) of
// s. r = (1, 0) leaves s unchanged bit for bit.
__device__ __forceinline__ Split turn(const Split& s, float2 r) {
    Split o;
    o.a = s.a;
    o.u = make_float3(__fmaf_rn(r.y, s.w.x, __fmul_rn(r.x, s.u.x)), __fmaf_rn(r.y, s.w.y, __fmul_rn(r.x, s.u.y)),
                      __fmaf_rn(r.y, s.w.z, __fmul_rn(r.x, s.u.z)));
    o.w = make_float3(__fmaf_rn(r.x, s.w.x, -__fmul_rn(r.y, s.u.x)), __fmaf_rn(r.x, s.w.y, -__fmul_rn(r.y, s.u.y)),
                      __fmaf_rn(r.x, s.w.z, -__fmul_rn(r.y, s.u.z)));
    return o;
}
__device__ __forceinline__ float3 place(const Split& s, float cs, float sn) {
    return make_float3(__fmaf_rn(sn, s.w.x, __fmaf_rn(cs, s.u.x, s.a.x)),
                       __fmaf_rn(sn, s.w.y, __fmaf_rn(cs, s.u.y, s.a.y)),
                       __fmaf_rn(sn, s.w.z, __fmaf_rn(cs, s.u.z, s.a.z)));
}

// Angle tables in shared memory are paired: entry p holds (cos, cos, sin, sin)
// of angles 2p and 2p+1, so two candidates' coordinates come from one packed
// FP32 multiply-add (the same rounding as two fmaf) per axis and term.
__device__ __forceinline__ float2 angle_at(const float4* t, int j) {
    const float4 v = t[j >> 1];
    return (j & 1) ? make_float2(v.y, v.w) : make_float2(v.x, v.z);
}
__device__ __forceinline__ float2 dup2(float v) { return make_float2(v, v); }
// Square root for the two pruning bounds only (never for a value that enters a result): x * rsqrt(x) is
// within about 2^-22 relative of sqrt(x), the order of the FP32 rounding already in x.
//  - circle bounds of the bump check: near the threshold (2 A = 4 grid units at h = 0.5 A) and for atoms
//    up to 2^8 grid units from the axis, (rho - r)^2 + (t - h)^2 moves by under 1e-3 grid^2, inside the
//    bound's 0.05 margin, so the same pairs go on to the per-angle tests;
//  - a moving atom's circle inside the padded box: its radius moves by under 1e-4 grid units, inside the
//    test's 1e-3 margin, so the unchecked lookup path is taken only where it is safe.
// Non-positive x (an atom on the axis) gives about 1e-15.
__device__ __forceinline__ float bound_sqrt(float x) {
    x = fmaxf(x, 1e-30f);
    return x * rsqrtf(x);
}

// Eq. 1's inner minimum taken over the probe points themselves, at grid
// position t shifted by +0.5 (points stored shifted alike), floored at 1.
__device__ __forceinline__ float exact_min(const PocketDev& pd, float3 t) {
    float m = 3.0e38f;
    for (int j = 0; j < pd.npts; ++j) {
        const float4 q = __ldg(pd.pts + j);
        const float dx = t.x - q.x, dy = t.y - q.y, dz = t.z - q.z;
        m = fminf(m, fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    }
    return fmaxf(m, 1.f);
}

// Field term of one atom at shifted grid position t.
// MODE 0 nearest (t shifted by +0.5: voxel = floor(t), inside iff 0 <= t < n)
// MODE 1 trilinear (unshifted: inside iff 0 <= t <= n-1)
// MODE 2 exact points (shifted as MODE 0, same inside test; no outside penalty:
//        the distance to the points is defined everywhere)
// Returns the term; *in reports whether the atom is inside the box. With
// CLIP the value is only meaningful when inside; without CLIP the lookup is
// clamped and the squared excess outside the box is added.
template <int MODE, bool CLIP>
__device__ __forceinline__ float term(const PocketDev& pd, const uint16_t* __restrict__ K, float3 t, bool* in) {
    if (MODE == 2) {
        *in = (vox(t.x) < (uint32_t)pd.nx) & (vox(t.y) < (uint32_t)pd.ny) & (vox(t.z) < (uint32_t)pd.nz);
        return exact_min(pd, t);
    } else if (MODE == 0) {
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

// Infeasible-candidate bits of one sweep phase, per lane: up to BW 64-bit
// words (448 candidates), lane-interleaved after the warp's coordinates; a
// run uses bw = ceil(largest phase / 64) of them.
constexpr int BW = 7;
// Besides its coordinate slice a warp keeps in shared memory only the bump
// bits (bw words per lane), the phase's candidate angles (64 bw, plus a
// chunk's worth of padding) and the sweep's atom-index lists (up to 258
// bytes; the area's last word holds the warp's count of gated lookups): the
// rest of the SM's shared memory serves as L1 cache for the field lookups.
constexpr int IDX_FLOATS = 68;
// per pose slot of the warp: its score (-1 if it started outside the box) while its lanes serve other
// poses (the remap of working poses onto more lanes, below)
constexpr int POSE_FLOATS = 32;
// Entries of the phase's angle table past 64 bw: a chunk's worth for the
// lookups, and the 12-candidate blocks of the bump tests.
__host__ __device__ constexpr int ptab_pad(int kc) { return kc > 12 ? kc : 12; }
__host__ __device__ constexpr int warp_extra_floats(int kc, int bw) {
    return bw * 64 + 2 * (64 * bw + ptab_pad(kc)) + IDX_FLOATS + POSE_FLOATS;
}
// every warp's area starts on a 16-byte boundary (the angle table is read as float4): slices are multiples
// of 4 floats, and so are these parts
static_assert(IDX_FLOATS % 4 == 0 && POSE_FLOATS % 4 == 0 && (2 * ptab_pad(8)) % 4 == 0 && (2 * ptab_pad(18)) % 4 == 0 &&
                  (2 * ptab_pad(36)) % 4 == 0,
              "per-warp shared-memory areas keep 16-byte alignment");

// 32-bit sums over the Q lanes of a pose.
__device__ __forceinline__ uint32_t group_add_u(uint32_t v, int Q) {
    for (int off = Q >> 1; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
    return v;
}
template <class M>
__device__ __forceinline__ M group_or(M v, int Q) {
    for (int off = Q >> 1; off > 0; off >>= 1) v |= __shfl_xor_sync(FULL, v, off);
    return v;
}

// Accumulator of one candidate: exact integers in nearest mode, floats in trilinear mode.
template <int MODE>
struct Acc {
    using T = uint32_t;
};
template <>
struct Acc<1> {
    using T = float;
};
template <>
struct Acc<2> {
    using T = float;
};

// Trilinear term (MODE 1) from the corner texture: the voxel floor(c) of the clamped position c is fetched
// at its centre, so the texel is the one the weights c - floor(c) refer to. At c = n - 1 exactly the
// repeated upper corners with weight 0 give the value the lower voxel gives with weight 1.
template <bool CLIP>
__device__ __forceinline__ float term_tri(const PocketDev& pd, float3 t, bool* in) {
    const float hx = (float)(pd.nx - 1), hy = (float)(pd.ny - 1), hz = (float)(pd.nz - 1);
    *in = (t.x >= 0.f) & (t.x <= hx) & (t.y >= 0.f) & (t.y <= hy) & (t.z >= 0.f) & (t.z <= hz);
    const float cx = fminf(fmaxf(t.x, 0.f), hx), cy = fminf(fmaxf(t.y, 0.f), hy), cz = fminf(fmaxf(t.z, 0.f), hz);
    const float x0 = floorf(cx), y0 = floorf(cy), z0 = floorf(cz);
    const float fx = cx - x0, fy = cy - y0, fz = cz - z0;
    const uint4 c = tex3D<uint4>(pd.Kc, x0 + 0.5f, y0 + 0.5f, z0 + 0.5f);
    const float c000 = (float)(c.x & 0xffffu), c100 = (float)(c.x >> 16), c010 = (float)(c.y & 0xffffu),
                c110 = (float)(c.y >> 16), c001 = (float)(c.z & 0xffffu), c101 = (float)(c.z >> 16),
                c011 = (float)(c.w & 0xffffu), c111 = (float)(c.w >> 16);
    const float c00 = fmaf(fx, c100 - c000, c000), c10 = fmaf(fx, c110 - c010, c010);
    const float c01 = fmaf(fx, c101 - c001, c001), c11 = fmaf(fx, c111 - c011, c011);
    const float c0 = fmaf(fy, c10 - c00, c00), c1 = fmaf(fy, c11 - c01, c01);
    const float v = fmaf(fz, c1 - c0, c0);
    if (CLIP) return v;
    const float ex = t.x - cx, ey = t.y - cy, ez = t.z - cz;
    return v + (ex * ex + ey * ey + ez * ez);
}

// Nearest-voxel value with the bounds test (shifted grid position t): the value
// of the voxel (clamped to the box when outside) and whether t is inside.
__device__ __forceinline__ uint32_t lookup_checked(const PocketDev& pd, const uint16_t* __restrict__ K, float3 t,
                                                   bool* in) {
    const uint32_t ix = vox(t.x), iy = vox(t.y), iz = vox(t.z);
    *in = (ix < (uint32_t)pd.nx) & (iy < (uint32_t)pd.ny) & (iz < (uint32_t)pd.nz);
    const int cx = min(max((int)ix, 0), pd.nx - 1), cy = min(max((int)iy, 0), pd.ny - 1),
              cz = min(max((int)iz, 0), pd.nz - 1);
    return __ldg(K + (cx + pd.nx * (cy + pd.ny * cz)));
}

// Squared distance outside the box of a shifted nearest-mode position.
__device__ __forceinline__ float outside2(const PocketDev& pd, float3 t) {
    const float ex = fmaxf(-t.x, 0.f) + fmaxf(t.x - (float)pd.nx, 0.f);
    const float ey = fmaxf(-t.y, 0.f) + fmaxf(t.y - (float)pd.ny, 0.f);
    const float ez = fmaxf(-t.z, 0.f) + fmaxf(t.z - (float)pd.nz, 0.f);
    return ex * ex + ey * ey + ez * ez;
}

// Candidates per block of the lookup gate: a block whose candidates are all
// infeasible for every pose of the warp is not scored.
__host__ __device__ constexpr int gate_block(int kc) { return kc % 6 == 0 ? 6 : 4; }

// Field terms of moving atoms at the chunk's KC angles, added to acc. The
// angles' (cos, sin) come from the warp's shared table (the same for every
// lane). fast: every circle lies inside the box, so no bounds tests. With
// CLIP an angle that puts an atom outside sets its bit in box; without CLIP
// the lookup is clamped and the squared distance outside goes to pen.
template <int KC, int MODE, bool CLIP, int NA>
__device__ __forceinline__ void score_atoms(const PocketDev& pd, const uint16_t* __restrict__ K,
                                            const Split (&s)[NA], bool fast, const float4* __restrict__ cst,
                                            typename Acc<MODE>::T (&acc)[KC], float (&pen)[KC], uint64_t& box,
                                            uint64_t need) {
    if (MODE == 0 && fast) {
        // padded field: circle centres moved by PAD voxels; outside values sum past OUTSIDE.
        // Candidates two at a time: packed multiply-adds place both, packed adds floor both.
        float2 ax[NA], ay[NA], az[NA], ux[NA], uy[NA], uz[NA], wx[NA], wy[NA], wz[NA];
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            ax[a] = dup2(s[a].a.x + (float)PAD);
            ay[a] = dup2(s[a].a.y + (float)PAD);
            az[a] = dup2(s[a].a.z + (float)PAD);
            ux[a] = dup2(s[a].u.x);
            uy[a] = dup2(s[a].u.y);
            uz[a] = dup2(s[a].u.z);
            wx[a] = dup2(s[a].w.x);
            wy[a] = dup2(s[a].w.y);
            wz[a] = dup2(s[a].w.z);
        }
        // blocks of candidates that no pose of the warp needs (all infeasible) are skipped
        constexpr int BLK = gate_block(KC);
        static_assert(KC % 2 == 0 && BLK % 2 == 0, "candidates go in pairs");
#pragma unroll
        for (int jb = 0; jb < KC; jb += BLK) {
            if ((need >> jb) & ((1ull << BLK) - 1ull)) {
#pragma unroll
                for (int j = jb; j < jb + BLK && j < KC; j += 2) {
                    const float4 cc = cst[j >> 1];
                    const float2 c2 = make_float2(cc.x, cc.y), s2 = make_float2(cc.z, cc.w);
#pragma unroll
                    for (int a = 0; a < NA; ++a) {
                        // a + cos u + sin w; the texture unit takes the floor and the voxel's address
                        const float2 tx = __ffma2_rn(s2, wx[a], __ffma2_rn(c2, ux[a], ax[a]));
                        const float2 ty = __ffma2_rn(s2, wy[a], __ffma2_rn(c2, uy[a], ay[a]));
                        const float2 tz = __ffma2_rn(s2, wz[a], __ffma2_rn(c2, uz[a], az[a]));
                        acc[j] += tex3D<unsigned>(pd.Kt, tx.x, ty.x, tz.x);
                        acc[j + 1] += tex3D<unsigned>(pd.Kt, tx.y, ty.y, tz.y);
                    }
                }
            }
        }
    } else if (MODE == 0) {
#pragma unroll
        for (int j = 0; j < KC; ++j) {
            const float2 c = angle_at(cst, j);
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                const float3 t = place(s[a], c.x, c.y);
                bool in;
                acc[j] += lookup_checked(pd, K, t, &in);
                if (!in) {
                    if (CLIP) box |= 1ull << j;
                    else pen[j] += outside2(pd, t);
                }
            }
        }
    } else if (MODE == 2) {
        // exact points: the chunk's positions stay in registers while the points stream by
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            float3 t[KC];
            float m[KC];
#pragma unroll
            for (int j = 0; j < KC; ++j) {
                const float2 c = angle_at(cst, j);
                t[j] = place(s[a], c.x, c.y);
                m[j] = 3.0e38f;
            }
            for (int p = 0; p < pd.npts; ++p) {
                const float4 q = __ldg(pd.pts + p);
#pragma unroll
                for (int j = 0; j < KC; ++j) {
                    const float dx = t[j].x - q.x, dy = t[j].y - q.y, dz = t[j].z - q.z;
                    m[j] = fminf(m[j], fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
                }
            }
#pragma unroll
            for (int j = 0; j < KC; ++j) {
                acc[j] += fmaxf(m[j], 1.f);
                const bool in = (vox(t[j].x) < (uint32_t)pd.nx) & (vox(t[j].y) < (uint32_t)pd.ny) &
                                (vox(t[j].z) < (uint32_t)pd.nz);
                if (CLIP && !in) box |= 1ull << j;
            }
        }
    } else {
        // blocks of candidates that no pose of the warp needs (all infeasible) are skipped
        constexpr int BLK = gate_block(KC);
#pragma unroll
        for (int jb = 0; jb < KC; jb += BLK) {
            if ((need >> jb) & ((1ull << BLK) - 1ull)) {
#pragma unroll
                for (int j = jb; j < jb + BLK && j < KC; j += 2) {
                    // two candidates per packed multiply-add (the roundings of place)
                    const float4 cc = cst[j >> 1];
                    const float2 c2 = make_float2(cc.x, cc.y), s2 = make_float2(cc.z, cc.w);
#pragma unroll
                    for (int a = 0; a < NA; ++a) {
                        const float2 tx = __ffma2_rn(s2, dup2(s[a].w.x), __ffma2_rn(c2, dup2(s[a].u.x), dup2(s[a].a.x)));
                        const float2 ty = __ffma2_rn(s2, dup2(s[a].w.y), __ffma2_rn(c2, dup2(s[a].u.y), dup2(s[a].a.y)));
                        const float2 tz = __ffma2_rn(s2, dup2(s[a].w.z), __ffma2_rn(c2, dup2(s[a].u.z), dup2(s[a].a.z)));
                        bool in0, in1;
                        acc[j] += term_tri<CLIP>(pd, make_float3(tx.x, ty.x, tz.x), &in0);
                        acc[j + 1] += term_tri<CLIP>(pd, make_float3(tx.y, ty.y, tz.y), &in1);
                        if (CLIP && !in0) box |= 1ull << j;
                        if (CLIP && !in1) box |= 2ull << j;
                    }
                }
            }
        }
    }
}

template <int KC, int MODE, bool CLIP>
__global__ void __launch_bounds__(256, KC <= 18 ? 2 : 1) sweep_kernel(SweepParams P) {
    extern __shared__ float smem[];
    using AT = typename Acc<MODE>::T;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    float* xs = smem + (size_t)warp * (P.slice + warp_extra_floats(KC, P.bw));
    unsigned long long* bump = reinterpret_cast<unsigned long long*>(xs + P.slice);  // [bw][32]
    float2* ptab = reinterpret_cast<float2*>(xs + P.slice + P.bw * 64);             // the phase's angles, paired
    uint8_t* sidx = reinterpret_cast<uint8_t*>(ptab + 64 * P.bw + ptab_pad(KC));    // the sweep's index lists
    unsigned long long* col = bump + lane;
    // the last word of the index-list area (lists take at most 258 bytes): the warp's count of
    // lookups left out by the gate in the current task
    unsigned* wlook = reinterpret_cast<unsigned*>(sidx) + (IDX_FLOATS - 1);
    float* smS = reinterpret_cast<float*>(sidx) + IDX_FLOATS;  // [32] pose scores (-1: not live)
    const float shift = MODE == 1 ? 0.0f : 0.5f;

    for (;;) {
        int task = 0;
        if (lane == 0) task = (int)atomicAdd(P.counter, 1u);
        task = __shfl_sync(FULL, task, 0);
        if (task >= P.ntask) break;
        const int2 tk = P.tasks[task];
        int lq = tk.y >> 16;
        int Q = 1 << lq;             // lanes per pose (they split the pose's atoms)
        const int G = 32 >> lq;      // poses of this warp (columns of its coordinate slice)
        int ps = lane >> lq;         // pose slot
        int q = lane & (Q - 1);
        const int pocket = tk.x / P.nlig, b = tk.x % P.nlig;
#ifdef GEODOCK_CHECKED
        if (!GD_OK(P.check, pocket < P.npockets, 7, pocket)) continue;
        {
            const LigDev Lc = P.lig[b];
            if (!GD_OK(P.check, Lc.atom_off >= 0 && Lc.atom_off + Lc.l <= P.natoms, 1, b)) continue;
            if (!GD_OK(P.check, 3 * Lc.l * G <= P.slice, 2, b)) continue;
        }
#endif
        const PocketDev& pd = P.pockets[pocket];
        const uint16_t* __restrict__ K = pd.K;
        const LigDev L = P.lig[b];
        const int p = (tk.y & 0xffff) * G + ps;
        bool active = p < P.n_poses;
        const float thr_g = (float)(P.bump_thr / pd.h);
        const float thr2 = thr_g * thr_g;
        const float nxf = (float)pd.nx, nyf = (float)pd.ny, nzf = (float)pd.nz;
        // circle inside [lo, hi) per axis: no per-angle bounds test needed. With clipping
        // the padded field flags outside positions by itself, so its padded box is enough.
        const float lo = (MODE == 0 && CLIP) ? -(float)PAD : 0.f;
        const float hix = MODE == 0 ? nxf - lo : nxf - 1.f, hiy = MODE == 0 ? nyf - lo : nyf - 1.f,
                    hiz = MODE == 0 ? nzf - lo : nzf - 1.f;

        // ---- initial rigid orientation, centroid on the pocket centre: the rotation (FP64) is
        // scaled to grid units once per pose, the atoms are placed in FP32
        {
            double R[9];
            pose_matrix(P.seed, L.id, active ? p : 0, R);
            const double ih = 1.0 / pd.h;
            float M[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) M[k] = (float)(R[k] * ih);
            const float ox = (float)((pd.centre[0] - pd.origin[0]) * ih + shift);
            const float oy = (float)((pd.centre[1] - pd.origin[1]) * ih + shift);
            const float oz = (float)((pd.centre[2] - pd.origin[2]) * ih + shift);
            const float gx = (float)L.g[0], gy = (float)L.g[1], gz = (float)L.g[2];
            for (int i = q; i < L.l; i += Q) {
                const float* x0 = P.xyz0 + 3 * (L.atom_off + i);
                const float d0 = x0[0] - gx, d1 = x0[1] - gy, d2 = x0[2] - gz;
                float3 t;
                t.x = fmaf(M[0], d0, fmaf(M[1], d1, fmaf(M[2], d2, ox)));
                t.y = fmaf(M[3], d0, fmaf(M[4], d1, fmaf(M[5], d2, oy)));
                t.z = fmaf(M[6], d0, fmaf(M[7], d1, fmaf(M[8], d2, oz)));
                st3(xs, i, G, ps, t);
            }
        }
        __syncwarp();
        float S_inc = 0.f;
        bool inbox = true;
        for (int i = q; i < L.l; i += Q) {
            bool in;
            S_inc += term<MODE, CLIP>(pd, K, ld3(xs, i, G, ps), &in);
            inbox = inbox && in;
        }
        S_inc = group_sum(S_inc, Q);
        inbox = group_all(inbox, Q);
        bool live = active && (!CLIP || inbox);
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

        // A pose whose last repetition committed no angle is at a fixed point: every further sweep
        // keeps its incumbent, so its sweeps are not computed (except when tracing); a warp
        // whose poses are all at a fixed point stops. nskip counts the pose-repetitions left out; a
        // pose that starts outside the box computes none.
        bool conv = !live;
        // pose-repetitions left out: with nearest-voxel values, counted for the warp (per repetition its
        // active poses less those computed, as poses move between lanes); otherwise by each pose's first
        // lane (the exact score's point loop runs slower with the warp-wide count: measured)
        const unsigned nact = (unsigned)max(0, min(G, P.n_poses - (tk.y & 0xffff) * G));
        unsigned nskip = 0;
        bool remapped = false;
        if (lane == 0) *wlook = 0u;
        if (__any_sync(FULL, live)) {
            for (int rep = 0; rep < P.repetitions; ++rep) {
                bool moved = false;  // did this pose commit any angle in this repetition
                const unsigned wm = __ballot_sync(FULL, live && !conv && q == 0);  // leaders of working poses
                const int nwork = __popc(wm);
                if (MODE == 0) nskip += nact - (unsigned)nwork;
                if (MODE == 0 && !P.trace_on && rep > 0) {
                    // The poses still working take over the lanes of those at a fixed point: each gets the
                    // most lanes (a power of two) that lets all of them fit the warp. A pose's coordinates
                    // stay in its slice column; its score moves with it. With nearest-voxel values every
                    // sum is an exact integer, so the results do not depend on the lanes a pose runs on.
                    int lqn = lq;
                    while (lqn < 5 && (nwork << (lqn + 1)) <= 32) ++lqn;
                    if (lqn > lq && nwork > 0) {
                        if (q == 0 && active) smS[ps] = live ? S_inc : -1.f;
                        const int j = lane >> lqn;
                        const bool asg = j < nwork;
                        unsigned mk = wm;  // the j-th working leader: drop the j lowest set bits
                        for (int t = 0; t < j && mk; ++t) mk &= mk - 1u;
                        const int leader = asg ? __ffs(mk) - 1 : 0;
                        const int psn = __shfl_sync(FULL, ps, leader);
                        const float Sn = __shfl_sync(FULL, S_inc, leader);
                        __syncwarp();
                        remapped = true;
                        lq = lqn;
                        Q = 1 << lq;
                        q = lane & (Q - 1);
                        ps = asg ? psn : 0;
                        S_inc = Sn;
                        active = asg;
                        live = asg;
                        conv = !asg;
                    }
                }
                const bool work = live && !conv;
                for (int si = 0; si < L.nside; ++si) {
                    const SideDev sd = P.side[L.side_off + si];
                    const int sweep = rep * L.nside + si;
                    const bool coarse =
                        P.coarse ? P.coarse[L.side_off + si] != 0 : (double)sd.m / (double)L.l <= P.threshold;
                    const bool peel = P.peel && !coarse;
                    // the sweep's index lists, staged in shared memory: M\{c}, then F\{b}, b, c
                    __syncwarp();
#ifdef GEODOCK_CHECKED
                    const bool lists_ok =
                        GD_OK(P.check, sd.nmov + sd.nfixS <= 4 * (IDX_FLOATS - 1), 3, L.side_off + si) &&
                        GD_OK(P.check, sd.mov_off >= 0 && sd.mov_off + sd.nmov <= P.nidx, 3, L.side_off + si) &&
                        GD_OK(P.check, sd.fix_off >= 0 && sd.fix_off + sd.nfixS <= P.nidx, 3, L.side_off + si) &&
                        GD_OK(P.check, sd.c < L.l && sd.b < L.l, 4, L.side_off + si);
                    if (!lists_ok) continue;  // the sweep is skipped (warp-uniform: one descriptor per warp)
                    for (int i = lane; i < sd.nmov + sd.nfixS; i += 32) {
                        const uint8_t a = P.idx[i < sd.nmov ? sd.mov_off + i : sd.fix_off + (i - sd.nmov)];
                        sidx[i] = GD_OK(P.check, a < L.l, 4, L.side_off + si) ? a : 0;
                    }
#else
                    for (int i = lane; i < sd.nmov + sd.nfixS; i += 32)
                        sidx[i] = P.idx[i < sd.nmov ? sd.mov_off + i : sd.fix_off + (i - sd.nmov)];
#endif
                    __syncwarp();
                    const uint8_t* mov = sidx;
                    const uint8_t* fix = sidx + sd.nmov;
                    const int nmov = sd.nmov, nfixB = sd.nfixB;
                    const int nslot = (nmov + Q - 1) / Q;  // moving atoms per lane (q + Q*s)
                    if (P.trace_on && active) {
                        const int64_t ci = (tbase + sweep) * P.tr.pmax;
                        float* tS = P.tr.cand_S + ci;
                        int* tSt = P.tr.cand_status + ci;
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
                    // fixed atoms' part of S: F plus the axis atom c. With nearest-voxel values and
                    // clipping, S_inc is the exact integer sum over the pose (inside the box), so when M
                    // is the smaller side its complement in S_inc is the same value, from fewer lookups.
                    float S_fix = 0.f;
                    if (MODE == 0 && CLIP && nmov < sd.nfixS) {
                        for (int i = q; i < nmov; i += Q) {
                            bool in;
                            S_fix += term<MODE, CLIP>(pd, K, ld3(xs, mov[i], G, ps), &in);
                        }
                        S_fix = S_inc - group_sum(S_fix, Q);
                    } else {
                        for (int i = q; i < sd.nfixS; i += Q) {
                            bool in;
                            S_fix += term<MODE, CLIP>(pd, K, ld3(xs, fix[i], G, ps), &in);
                        }
                        S_fix = group_sum(S_fix, Q);
                    }

                    unsigned long long best = make_key(S_inc, 0);
                    const int phases = peel ? 2 : 1;
                    int tile_first = 0;
                    bool have_tile = true;  // a pose with no feasible tile centre keeps its incumbent
                    float2 pre = make_float2(1.f, 0.f);  // angle origin of this pose's candidates
                    for (int ph = 0; ph < phases; ++ph) {
                        // candidates tab[j], j < ncand, in trace slots slot0 + j
                        int ncand, slot0;
                        const float2* tab;
                        if (!peel) {
                            ncand = (coarse ? P.P_lp : P.P_hp) - 1;
                            tab = (coarse ? P.cs_lp : P.cs_hp) + 1;
                            slot0 = 1;
                        } else if (ph == 0) {
                            ncand = P.n_tiles;
                            tab = P.cs_peel;
                            slot0 = 1;
                        } else {
                            // the tile's angles relative to its start, the same for every pose;
                            // each pose turns its circles to its own tile start (pre)
                            ncand = P.per_tile;
                            tab = P.cs_hp;
                            slot0 = 1 + P.n_tiles;
                        }

                        // ---- bump check for the whole phase. The closest approach of fixed atom y
                        // to the circle of moving atom x is sqrt((rho_y - r_x)^2 + (h_y - h_x)^2)
                        // (rho: distance from the axis, h: position along it); pairs that come within
                        // the threshold get the arc of angles where they do marked.
#ifdef GEODOCK_CHECKED
                        if (!GD_OK(P.check, ncand <= 64 * P.bw, 5, ncand)) ncand = 64 * P.bw;
#endif
                        const int nw = (ncand + 63) >> 6;
                        for (int w = 0; w < nw; ++w) col[w * 32] = 0ull;
                        // the phase's angles, the same for every lane; (1, 0) past the end
                        __syncwarp();
                        for (int j = lane; j < 64 * P.bw + ptab_pad(KC); j += 32) {
                            const float2 v = j < ncand ? tab[j] : make_float2(1.f, 0.f);
                            float* e = reinterpret_cast<float*>(ptab) + 4 * (j >> 1) + (j & 1);
                            e[0] = v.x;
                            e[2] = v.y;
                        }
                        __syncwarp();
                        {
                            const float lim = thr2 + 0.05f;  // margin over the FP32 error of the bound
                            // a moving side of at most 8 atoms: every lane of a pose holds all of them and the
                            // pose's lanes split the fixed atoms instead (not with the exact score, whose point
                            // loop runs slower in that build: measured)
                            const bool small = MODE != 2 && nmov <= 8;
                            const int nsl = small ? nmov : nslot;
                            for (int s0 = 0; s0 < nsl; s0 += 8) {
                                float r[8], h[8];
#pragma unroll
                                for (int j = 0; j < 8; ++j) {
                                    const int im = small ? s0 + j : q + Q * (s0 + j);
                                    r[j] = 1e18f;  // no atom: never close (its square stays finite)
                                    h[j] = 0.f;
                                    if (s0 + j < nsl && im < nmov) {
                                        float3 x = ld3(xs, mov[im], G, ps);
                                        float vx = x.x - gc.x, vy = x.y - gc.y, vz = x.z - gc.z;
                                        float t = kax.x * vx + kax.y * vy + kax.z * vz;
                                        r[j] = bound_sqrt(vx * vx + vy * vy + vz * vz - t * t);
                                        h[j] = t;
                                    }
                                }
                                // fixed atoms two at a time (independent loads in flight)
                                for (int f = small ? 2 * q : 0; f < nfixB; f += small ? 2 * Q : 2) {
                                    const int f1 = f + 1 < nfixB ? f + 1 : f;
                                    const float3 y0 = ld3(xs, fix[f], G, ps), y1 = ld3(xs, fix[f1], G, ps);
                                    unsigned near0 = 0, near1 = 0;
                                    {
                                        const float wx = y0.x - gc.x, wy = y0.y - gc.y, wz = y0.z - gc.z;
                                        const float t0 = kax.x * wx + kax.y * wy + kax.z * wz;
                                        const float rho0 = bound_sqrt(wx * wx + wy * wy + wz * wz - t0 * t0);
                                        const float vx = y1.x - gc.x, vy = y1.y - gc.y, vz = y1.z - gc.z;
                                        const float t1 = kax.x * vx + kax.y * vy + kax.z * vz;
                                        const float rho1 = bound_sqrt(vx * vx + vy * vy + vz * vz - t1 * t1);
                                        // two moving atoms per packed operation: (rho - r)^2 + (t - h)^2 with the
                                        // roundings of the scalar form (a subtraction is the addition of the negation)
                                        const float2 R0 = dup2(rho0), T0 = dup2(t0), R1 = dup2(rho1), T1 = dup2(t1);
#pragma unroll
                                        for (int j = 0; j < 8; j += 2) {
                                            if (j >= nsl - s0) break;  // the block's empty slots (warp-uniform)
                                            const float2 nr = make_float2(-r[j], -r[j + 1]), nh = make_float2(-h[j], -h[j + 1]);
                                            const float2 dr0 = __fadd2_rn(R0, nr), dh0 = __fadd2_rn(T0, nh);
                                            const float2 dr1 = __fadd2_rn(R1, nr), dh1 = __fadd2_rn(T1, nh);
                                            const float2 q0 = __ffma2_rn(dr0, dr0, __fmul2_rn(dh0, dh0));
                                            const float2 q1 = __ffma2_rn(dr1, dr1, __fmul2_rn(dh1, dh1));
                                            if (q0.x < lim) near0 |= 1u << j;
                                            if (q0.y < lim) near0 |= 2u << j;
                                            if (q1.x < lim) near1 |= 1u << j;
                                            if (q1.y < lim) near1 |= 2u << j;
                                        }
                                    }
                                    if (!work || !have_tile) near0 = 0;
                                    if (!work || !have_tile || f1 == f) near1 = 0;
                                    unsigned long long pairs = near0 | ((unsigned long long)near1 << 8);
                                    while (pairs) {
                                        const int e = __ffsll(pairs) - 1;
                                        pairs &= pairs - 1;
                                        const float3 y = e < 8 ? y0 : y1;
                                        const Split sp0 = split(ld3(xs, mov[small ? s0 + (e & 7) : q + Q * (s0 + (e & 7))], G, ps), gc, kax);
                                        const Split sp = peel ? turn(sp0, pre) : sp0;
                                        // d^2(theta) = A + B cos(theta) + C sin(theta) at every candidate
                                        const float dx = sp.a.x - y.x, dy = sp.a.y - y.y, dz = sp.a.z - y.z;
                                        const float A = dx * dx + dy * dy + dz * dz +
                                                        (sp.u.x * sp.u.x + sp.u.y * sp.u.y + sp.u.z * sp.u.z);
                                        const float B = 2.f * (dx * sp.u.x + dy * sp.u.y + dz * sp.u.z);
                                        const float C = 2.f * (dx * sp.w.x + dy * sp.w.y + dz * sp.w.z);
                                        // candidates 12 at a time, two per packed multiply-add; a block
                                        // may straddle two 64-bit words
                                        const float4* tw = reinterpret_cast<const float4*>(ptab);
                                        // the test is the sign bit of (A - thr^2) + B cos + C sin (FP32, two
                                        // candidates per packed multiply-add); the bits are shifted in from the
                                        // block's last candidate down to its first
                                        const float2 A2 = dup2(A - thr2), B2 = dup2(B), C2 = dup2(C);
                                        for (int g = 0; g < ncand; g += 12) {
                                            unsigned m12 = 0;
#pragma unroll
                                            for (int k = 5; k >= 0; --k) {
                                                const float4 t = tw[(g >> 1) + k];
                                                const float2 d2 = __ffma2_rn(C2, make_float2(t.z, t.w),
                                                                             __ffma2_rn(B2, make_float2(t.x, t.y), A2));
                                                m12 = __funnelshift_l(__float_as_uint(d2.y), m12, 1);
                                                m12 = __funnelshift_l(__float_as_uint(d2.x), m12, 1);
                                            }
                                            const int w = g >> 6, sh = g & 63;
                                            col[w * 32] |= (unsigned long long)m12 << sh;
                                            if (sh > 52 && w + 1 < P.bw && (m12 >> (64 - sh)))
                                                col[(w + 1) * 32] |= (unsigned long long)(m12 >> (64 - sh));
                                        }
                                    }
                                }
                            }
                        }

                        unsigned long long pbest = ~0ull;
                        for (int j0 = 0; j0 < ncand; j0 += KC) {
                            // the chunk's angles are the same for every lane of the warp
                            const int nvalid = min(KC, ncand - j0);
                            const float4* cst = reinterpret_cast<const float4*>(ptab) + (j0 >> 1);
                            AT acc[KC];
                            float pen[KC];
#pragma unroll
                            for (int j = 0; j < KC; ++j) {
                                acc[j] = (AT)0;
                                pen[j] = 0.f;
                            }
                            uint64_t box = 0ull;
                            // candidates of this chunk that some pose of the warp may still take
                            uint64_t need;
                            {
                                const int w = j0 >> 6, sh = j0 & 63;
                                uint64_t b0 = col[w * 32] >> sh;
                                if (sh + KC > 64 && w + 1 < P.bw) b0 |= col[(w + 1) * 32] << (64 - sh);
                                b0 = group_or(b0, Q);
                                uint64_t nd = (work && have_tile) ? ~b0 : 0ull;
                                nd &= nvalid >= 64 ? ~0ull : ((1ull << nvalid) - 1ull);
                                const unsigned lo = __reduce_or_sync(FULL, (unsigned)nd);
                                const unsigned hi = __reduce_or_sync(FULL, (unsigned)(nd >> 32));
                                need = ((uint64_t)hi << 32) | lo;
                            }

                            auto circle_inside = [&](const Split& sp) {
                                const float rad = bound_sqrt(sp.u.x * sp.u.x + sp.u.y * sp.u.y + sp.u.z * sp.u.z) + 1e-3f;
                                return sp.a.x - rad >= lo && sp.a.x + rad < hix && sp.a.y - rad >= lo &&
                                       sp.a.y + rad < hiy && sp.a.z - rad >= lo && sp.a.z + rad < hiz;
                            };
                            // one moving atom per pass: a single copy of the unrolled lookups keeps the hot
                            // code small enough for the instruction cache at two CTAs per SM
                            int s = 0;
                            for (; s < nslot; ++s) {
                                const int i0 = q + Q * s;
                                const bool h0 = i0 < nmov;
                                const Split one0 = split(ld3(xs, mov[h0 ? i0 : 0], G, ps), gc, kax);
                                Split one[1] = {peel ? turn(one0, pre) : one0};
                                const bool fast = __all_sync(FULL, !h0 || !work || circle_inside(one[0]));
                                // a pose not computed in this repetition makes no lookups (its lane idles)
                                if (h0 && work) score_atoms<KC, MODE, CLIP, 1>(pd, K, one, fast, cst, acc, pen, box, need);
                            }
                            // lookups left out by the gate: the valid candidates of blocks no pose needed,
                            // for every moving atom of every working pose (counted as if every pass took
                            // the fast path; the checked path scores all candidates, so this count is
                            // never below the lookups actually left out)
                            if (MODE != 2 && P.lookups_skipped) {
                                const unsigned nw = __popc(__ballot_sync(FULL, work && q == 0));
                                constexpr int BLK = gate_block(KC);
                                const uint64_t vm = nvalid >= 64 ? ~0ull : ((1ull << nvalid) - 1ull);
                                unsigned gone = 0;
#pragma unroll
                                for (int jb = 0; jb < KC; jb += BLK) {
                                    const uint64_t m = (((1ull << BLK) - 1ull) << jb) & vm;
                                    if (!(need & m)) gone += (unsigned)__popcll(m);
                                }
                                if (lane == 0 && gone && nw) *wlook += gone * (unsigned)nmov * nw;
                            }
                            // this chunk's bump bits
                            uint64_t bad;
                            {
                                const int w = j0 >> 6, sh = j0 & 63;
                                bad = col[w * 32] >> sh;
                                if (sh + KC > 64 && w + 1 < P.bw) bad |= col[(w + 1) * 32] << (64 - sh);
                            }
                            // combine the pose's lanes: every lane then holds the pose's full values
                            bad = group_or(bad, Q);
                            if (CLIP) box = group_or(box, Q);
#pragma unroll
                            for (int j = 0; j < KC; ++j) {
                                if (MODE == 0) acc[j] = (AT)group_add_u((uint32_t)acc[j], Q);
                                else acc[j] = (AT)group_sum((float)acc[j], Q);
                                if (!CLIP) pen[j] = group_sum(pen[j], Q);
                            }
#pragma unroll
                            for (int j = 0; j < KC; ++j) {
                                const float S = S_fix + (float)acc[j] + (CLIP ? 0.f : pen[j]);
                                const bool ok = j < nvalid && have_tile && !((bad >> j) & 1ull) &&
                                                !(CLIP && (((box >> j) & 1ull) || (MODE == 0 && (uint32_t)acc[j] >= OUTSIDE)));
                                const unsigned long long key = make_key(S, slot0 + j0 + j);
                                pbest = (ok && key < pbest) ? key : pbest;
                            }
                            if (P.trace_on && active && q == 0) {
                                // trace: every evaluated candidate's S and status
                                const int64_t ci = (tbase + sweep) * P.tr.pmax;
                                float* tS = P.tr.cand_S + ci;
                                int* tSt = P.tr.cand_status + ci;
#pragma unroll 1
                                for (int j = 0; j < nvalid; ++j) {
                                    if (!have_tile) break;
                                    float accj = 0.f, penj = 0.f;
                                    bool outj = false;
#pragma unroll
                                    for (int i = 0; i < KC; ++i)
                                        if (i == j) {
                                            accj = (float)acc[i];
                                            penj = CLIP ? 0.f : pen[i];
                                            outj = MODE == 0 && (uint32_t)acc[i] >= OUTSIDE;
                                        }
                                    const bool clash = (bad >> j) & 1ull;
                                    const bool out = CLIP && (((box >> j) & 1ull) || outj);
                                    tS[slot0 + j0 + j] = S_fix + accj + penj;
                                    tSt[slot0 + j0 + j] = clash ? 0 : (out ? -1 : 1);
                                }
                            }
                        }
                        if (peel && ph == 0) {
                            // the best tile centre picks the tile; its angles are the next phase
                            have_tile = pbest != ~0ull;
                            const int t = have_tile ? (int)(pbest & 0xffffffffu) - 1 : 0;
                            tile_first = t * P.per_tile;
                            pre = P.cs_hp[tile_first];
                        } else {
                            best = pbest < best ? pbest : best;
                        }
                    }
                    const int kb = work ? (int)(best & 0xffffffffu) : 0;
                    if (kb != 0) {
                        // the same rotation as the candidate's evaluation
                        const float2 v = !peel ? (coarse ? P.cs_lp : P.cs_hp)[kb] : P.cs_hp[kb - 1 - P.n_tiles];
                        const float2 r0 = !peel ? make_float2(1.f, 0.f) : pre;
                        for (int s = 0; s < nslot; ++s) {
                            const int im = q + Q * s;
                            if (im < nmov) {
                                const int i = mov[im];
                                st3(xs, i, G, ps, place(turn(split(ld3(xs, i, G, ps), gc, kax), r0), v.x, v.y));
                            }
                        }
                        S_inc = __uint_as_float((unsigned)(best >> 32));
                    }
                    if (P.trace_on && active && q == 0) P.tr.chosen_k[tbase + sweep] = kb;
                    moved = moved || kb != 0;
                    __syncwarp();
                }
                // a repetition in which no pose of the warp moved left every pose where it was, so
                // each further repetition would repeat it exactly: stop (the trace records them all)
                if (MODE != 0 && conv && active && q == 0) ++nskip;
                if (!P.trace_on && !moved) conv = true;
                if (!P.trace_on && !__any_sync(FULL, moved)) {
                    if (MODE == 0) nskip += (unsigned)(P.repetitions - 1 - rep) * nact;
                    else if (active && q == 0) nskip += (unsigned)(P.repetitions - 1 - rep);
                    break;
                }
            }
        } else {
            if (MODE == 0) nskip = (unsigned)P.repetitions * nact;
            else if (active && q == 0) nskip = (unsigned)P.repetitions;
        }
        if (remapped) {
            // every pose back in its own lanes, with its score
            if (q == 0 && active) smS[ps] = live ? S_inc : -1.f;
            __syncwarp();
            lq = tk.y >> 16;
            Q = 1 << lq;
            ps = lane >> lq;
            q = lane & (Q - 1);
            active = (tk.y & 0xffff) * G + ps < P.n_poses;
            const float sv = active ? smS[ps] : -1.f;
            live = sv >= 0.f;
            S_inc = sv;
        }
        if (MODE != 0) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) nskip += __shfl_xor_sync(FULL, nskip, o);
        }
        if (P.skipped && lane == 0 && nskip) atomicAdd(P.skipped + tk.x, nskip);
        if (P.lookups_skipped && lane == 0 && *wlook) atomicAdd(P.lookups_skipped, (unsigned long long)*wlook);
        // ---- per-pose result
        if (active && q == 0 &&
            GD_OK(P.check, (int64_t)tk.x < (int64_t)P.npockets * P.nlig && p < P.n_poses, 6, tk.x)) {
            const int64_t pi = (int64_t)tk.x * P.n_poses + p;
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
                const int64_t ti = (int64_t)b * P.n_poses + p;
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
static __global__ void finalize_kernel(FinalParams F) {
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
static __global__ void field_kernel(uint16_t* K, int nx, int ny, int nz, const int4* pts, int npts) {
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
// Padded copy of the field: PAD voxels of OUTSIDE around the grid.
static __global__ void corner_field_kernel(uint4* Kc, const uint16_t* K, int nx, int ny, int nz) {
    const int64_t n = (int64_t)nx * ny * nz;
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((int64_t)nx * ny));
    const int x1 = x + 1 < nx ? x + 1 : x, y1 = y + 1 < ny ? y + 1 : y, z1 = z + 1 < nz ? z + 1 : z;
    auto at = [&](int i, int j, int l) { return (uint32_t)K[((int64_t)l * ny + j) * nx + i]; };
    Kc[v] = make_uint4(at(x, y, z) | (at(x1, y, z) << 16), at(x, y1, z) | (at(x1, y1, z) << 16),
                       at(x, y, z1) | (at(x1, y, z1) << 16), at(x, y1, z1) | (at(x1, y1, z1) << 16));
}

static __global__ void pad_field_kernel(uint32_t* Kp, const uint16_t* K, int nx, int ny, int nz) {
    const int pnx = nx + 2 * PAD, pny = ny + 2 * PAD, pnz = nz + 2 * PAD;
    const int64_t n = (int64_t)pnx * pny * pnz;
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int x = (int)(v % pnx) - PAD, y = (int)((v / pnx) % pny) - PAD, z = (int)(v / ((int64_t)pnx * pny)) - PAD;
    const bool in = x >= 0 && y >= 0 && z >= 0 && x < nx && y < ny && z < nz;
    Kp[v] = in ? (uint32_t)K[(int64_t)z * ny * nx + (int64_t)y * nx + x] : OUTSIDE;
}
#endif  // GD_DEFINE_AUX_KERNELS

}  // namespace gd
