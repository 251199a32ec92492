// Device code of the local refinement stage and of the differentiable score
// (not in the paper, which only mentions steepest descent; the adjoint
// follows from Eq. 1 with a trilinear field).
//
// Pose degrees of freedom q = (t, omega, theta_1..theta_T): the torsion deltas
// turn, for every rotatable bond, the side away from atom 0 about the axis
// b -> c (c on the moving side), deepest bond first; then the pose rotates by
// the rotation vector omega about the centroid g of its input coordinates and
// moves by t:  z = g + R(omega) (tau(x) - g) + t.
//
// Score: S = sum_i D(z_i) with D the trilinear interpolant of the floored
// field K (grid units; D at the clamped position, plus the squared excess
// outside the box when clipping is off), o = l / (h^2 S).
//
// Adjoint (reverse mode): with p_i = d f / d z_i,
//   d f / d t       = sum_i p_i
//   d f / d omega   = J(omega)^T sum_i (z_i - g - t) x p_i,
//                     J = I + (1 - cos a)/a^2 [w]x + (a - sin a)/a^3 [w]x^2, a = |w|
//                     (left Jacobian of the exponential map)
//   d f / d theta_k = axis_k . sum_{i in M_k} (z_i - z_c) x p_i, axis and c in z.
//
// One warp owns one ligand (or one (pocket, ligand) pair); lanes walk its
// atoms. Coordinates live in shared memory as [atom][xyz] (Å).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "geodock_kernels.cuh"

namespace gd {

// A refinement torsion: the fragment-sweep descriptor of the side away from
// atom 0, and the torsion's slot in q (the ligand's rotatable-bond order).
struct RefTorDev {
    int side;  // index into the batch's SideDev array
    int k;     // q[6 + k]
};

struct RefLigDev {
    int tor_off;    // first RefTorDev, application order (deepest bond first)
    int T;          // torsions
    int check_off;  // first word of the bump-pair rows: l rows of wpr words, bit j of row i: pair (i, j)
    int wpr;
};

// Step-length rule of the refinement: the largest first-order atom
// displacement of a step starts at LAMBDA0 Å, grows by GROW after an
// accepted step (at most LAMBDA_MAX) and shrinks by SHRINK after a rejected one.
constexpr float REFINE_LAMBDA0 = 0.25f, REFINE_LAMBDA_MAX = 1.0f, REFINE_GROW = 1.5f, REFINE_SHRINK = 0.5f;

// Sizes of a batch's arrays, for the index checks of checked builds (GEODOCK_CHECKED; see GD_OK).
struct BatchBounds {
    int natoms, nside, nidx, ntor, nchk, lmax;
    unsigned long long* check;  // status word of the checks (nullable)
};

struct RefineTraceDev {
    int gstride;        // 6 + largest T
    float* G;           // [pair][step][gstride]
    float* D;           // [pair][step]
    float* lam;
    float* S_new;
    int32_t* verdict;   // bit0 S_new < S, bit1 bump-free, bit2 inside the box
    int32_t* accept;
    float* S_start;     // [pair]
    float* S_final;
    int32_t* status;    // 0 refined, 1 skipped
};

struct RefineParams {
    const LigDev* lig;
    const SideDev* side;
    const uint8_t* idx;
    const RefLigDev* rlig;
    const RefTorDev* rtor;
    const uint32_t* check;
    const PocketDev* pockets;
    int npairs, nlig, natoms;
    int steps, clip;
    float thr2;           // bump threshold squared, Å^2
    const float* xyz_in;  // Å, ((pocket * natoms + atom_off) + i) * 3
    float* xyz_out;       // same layout
    float* result;        // dock_result words per pair: score, pose (-1), status, reserved
    int trace_on;
    RefineTraceDev tr;
    BatchBounds bounds;
};

// Differentiable-score launches: one warp per ligand of a batch.
struct ScoreParams {
    const LigDev* lig;
    const SideDev* side;
    const uint8_t* idx;
    const RefLigDev* rlig;
    const RefTorDev* rtor;
    const PocketDev* pocket;  // device pointer to one pocket
    int nlig, clip, qstride;
    const float* x;       // input coordinates, Å, atom_off layout
    const float* q;       // [ligand][qstride]
    const float* grad_in; // score backward: d L / d o per ligand (nullable: ones); dof backward: d L / d z
    float* out;           // o per ligand / z / grad
    BatchBounds bounds;
};

// ----------------------------------------------------------------- helpers

__device__ __forceinline__ float wsum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}
__device__ __forceinline__ float wmax(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(FULL, v, o));
    return v;
}
__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 add3(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 sub3(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 mul3(float3 a, float s) { return f3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 lds3(const float* s, int i) { return f3(s[3 * i], s[3 * i + 1], s[3 * i + 2]); }
__device__ __forceinline__ void sts3(float* s, int i, float3 v) {
    s[3 * i] = v.x;
    s[3 * i + 1] = v.y;
    s[3 * i + 2] = v.z;
}
__device__ __forceinline__ float3 wsum3(float3 v) { return f3(wsum(v.x), wsum(v.y), wsum(v.z)); }

// Rodrigues rotation of x by the angle with cosine ct and sine st about the
// unit axis k through c.
__device__ __forceinline__ float3 rot_about(float3 x, float3 c, float3 k, float ct, float st) {
    const float3 v = sub3(x, c);
    const float kv = dot3(k, v);
    return add3(c, add3(add3(mul3(v, ct), mul3(cross3(k, v), st)), mul3(k, kv * (1.f - ct))));
}

// Rotation matrix of the rotation vector w (Rodrigues' formula).
__device__ __forceinline__ void expmap3(float3 w, float R[9]) {
    const float th = sqrtf(dot3(w, w));
    if (th == 0.f) {
        R[0] = R[4] = R[8] = 1.f;
        R[1] = R[2] = R[3] = R[5] = R[6] = R[7] = 0.f;
        return;
    }
    const float3 k = mul3(w, 1.f / th);
    float s, c;
    sincosf(th, &s, &c);
    const float C = 1.f - c;
    R[0] = c + k.x * k.x * C;
    R[1] = k.x * k.y * C - k.z * s;
    R[2] = k.x * k.z * C + k.y * s;
    R[3] = k.y * k.x * C + k.z * s;
    R[4] = c + k.y * k.y * C;
    R[5] = k.y * k.z * C - k.x * s;
    R[6] = k.z * k.x * C - k.y * s;
    R[7] = k.z * k.y * C + k.x * s;
    R[8] = c + k.z * k.z * C;
}

// J(w)^T v for the left Jacobian of the exponential map.
__device__ __forceinline__ float3 jl_transpose(float3 w, float3 v) {
    const float a2 = dot3(w, w), a = sqrtf(a2);
    float A, B;
    if (a < 1e-2f) {
        A = 0.5f - a2 * (1.f / 24.f);
        B = 1.f / 6.f - a2 * (1.f / 120.f);
    } else {
        float s, c;
        sincosf(a, &s, &c);
        A = (1.f - c) / a2;
        B = (a - s) / (a2 * a);
    }
    const float3 wv = cross3(w, v), wwv = cross3(w, wv);
    return add3(sub3(v, mul3(wv, A)), mul3(wwv, B));
}

// Trilinear term (grid units) of the floored field at Å position z, with its
// gradient d D / d z (grid units per Å) and the inside flag (0 <= t <= n-1).
__device__ __forceinline__ float tri_term(const PocketDev& pd, float3 o, float inv_h, float3 z, bool clip, float3* dD,
                                          bool* inside) {
    const float t[3] = {(z.x - o.x) * inv_h, (z.y - o.y) * inv_h, (z.z - o.z) * inv_h};
    const int n[3] = {pd.nx, pd.ny, pd.nz};
    float tc[3], f[3], ex[3];
    int i0[3];
    bool in = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float hi = (float)(n[a] - 1);
        tc[a] = fminf(fmaxf(t[a], 0.f), hi);
        ex[a] = t[a] - tc[a];
        in = in && ex[a] == 0.f;
        i0[a] = min((int)floorf(tc[a]), n[a] - 2);
        f[a] = tc[a] - (float)i0[a];
    }
    const int64_t base = ((int64_t)i0[2] * n[1] + i0[1]) * n[0] + i0[0];
    const int64_t sy = n[0], sz = (int64_t)n[0] * n[1];
    float k[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) k[c] = (float)__ldg(pd.K + base + (c & 1) + ((c >> 1) & 1) * sy + (c >> 2) * sz);
    // interpolate along x, then y, then z
    const float x00 = k[0] + f[0] * (k[1] - k[0]), x10 = k[2] + f[0] * (k[3] - k[2]);
    const float x01 = k[4] + f[0] * (k[5] - k[4]), x11 = k[6] + f[0] * (k[7] - k[6]);
    const float y0 = x00 + f[1] * (x10 - x00), y1 = x01 + f[1] * (x11 - x01);
    float D = y0 + f[2] * (y1 - y0);
    // derivatives of the same interpolant
    const float dx0 = (k[1] - k[0]) + f[1] * ((k[3] - k[2]) - (k[1] - k[0]));
    const float dx1 = (k[5] - k[4]) + f[1] * ((k[7] - k[6]) - (k[5] - k[4]));
    float g[3] = {dx0 + f[2] * (dx1 - dx0), (x10 - x00) + f[2] * ((x11 - x01) - (x10 - x00)), y1 - y0};
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if (ex[a] != 0.f) g[a] = clip ? 0.f : 2.f * ex[a];
    if (!clip) D += ex[0] * ex[0] + ex[1] * ex[1] + ex[2] * ex[2];
    *dD = f3(g[0] * inv_h, g[1] * inv_h, g[2] * inv_h);
    *inside = in;
    return D;
}

// Pocket frame in FP32.
struct Frame {
    float3 o;
    float inv_h, h2;
};
__device__ __forceinline__ Frame frame_of(const PocketDev& pd) {
    Frame F;
    F.o = f3((float)pd.origin[0], (float)pd.origin[1], (float)pd.origin[2]);
    F.inv_h = (float)(1.0 / pd.h);
    F.h2 = (float)(pd.h * pd.h);
    return F;
}

// S of the warp's pose z (shared memory) and the inside flag; with dS given,
// also d S / d z_i into dS (shared memory, [atom][xyz]).
__device__ __forceinline__ float warp_score(const PocketDev& pd, const Frame& F, const float* z, int l, bool clip,
                                           float* dS, bool* inside) {
    const int lane = threadIdx.x & 31;
    float S = 0.f;
    bool in = true;
    for (int i = lane; i < l; i += 32) {
        float3 d;
        bool ii;
        S += tri_term(pd, F.o, F.inv_h, lds3(z, i), clip, &d, &ii);
        in = in && ii;
        if (dS) sts3(dS, i, d);
    }
    *inside = __all_sync(FULL, in);
    return wsum(S);
}

// Applies the torsion deltas th(k) (deepest bond first) to the warp's pose y in place.
template <class TH>
__device__ __forceinline__ void warp_torsions(const SideDev* side, const uint8_t* idx, const LigDev& L,
                                              const RefLigDev& R, const RefTorDev* rtor, float* y, TH th) {
    const int lane = threadIdx.x & 31;
    for (int e = 0; e < R.T; ++e) {
        const RefTorDev rt = rtor[R.tor_off + e];
        const SideDev sd = side[L.side_off + rt.side];
        const float a = th(rt.k);
        if (a == 0.f) continue;
        const float3 c = lds3(y, sd.c);
        float3 k = sub3(c, lds3(y, sd.b));
        k = mul3(k, rsqrtf(dot3(k, k)));
        float s, co;
        sincosf(a, &s, &co);
        __syncwarp();
        for (int j = lane; j < sd.nmov; j += 32) {
            const int i = idx[sd.mov_off + j];
            sts3(y, i, rot_about(lds3(y, i), c, k, co, s));
        }
        __syncwarp();
    }
}

// Centroid of the warp's pose.
__device__ __forceinline__ float3 warp_centroid(const float* x, int l) {
    const int lane = threadIdx.x & 31;
    float3 g = f3(0.f, 0.f, 0.f);
    for (int i = lane; i < l; i += 32) g = add3(g, lds3(x, i));
    g = wsum3(g);
    return mul3(g, 1.f / (float)l);
}

// z = g + R(w)(y - g) + t in place (g precomputed from the input pose).
__device__ __forceinline__ void warp_rigid(float* y, int l, float3 g, float3 t, float3 w) {
    const int lane = threadIdx.x & 31;
    float R[9];
    expmap3(w, R);
    __syncwarp();
    for (int i = lane; i < l; i += 32) {
        const float3 v = sub3(lds3(y, i), g);
        sts3(y, i, f3(g.x + R[0] * v.x + R[1] * v.y + R[2] * v.z + t.x, g.y + R[3] * v.x + R[4] * v.y + R[5] * v.z + t.y,
                      g.z + R[6] * v.x + R[7] * v.y + R[8] * v.z + t.z));
    }
    __syncwarp();
}

// d f / d q at the pose z = apply(x, q) given p = d f / d z (shared memory):
// writes G[0..6+T) through put(k, value) (lane 0).
template <class PUT>
__device__ __forceinline__ void warp_dof_grad(const SideDev* side, const uint8_t* idx, const LigDev& L,
                                              const RefLigDev& R, const RefTorDev* rtor, const float* z,
                                              const float* p, float3 g, float3 t, float3 w, PUT put) {
    const int lane = threadIdx.x & 31;
    float3 gt = f3(0.f, 0.f, 0.f), tau = f3(0.f, 0.f, 0.f);
    for (int i = lane; i < L.l; i += 32) {
        const float3 pi = lds3(p, i);
        gt = add3(gt, pi);
        tau = add3(tau, cross3(sub3(sub3(lds3(z, i), g), t), pi));
    }
    gt = wsum3(gt);
    tau = wsum3(tau);
    const float3 gw = jl_transpose(w, tau);
    if (lane == 0) {
        put(0, gt.x);
        put(1, gt.y);
        put(2, gt.z);
        put(3, gw.x);
        put(4, gw.y);
        put(5, gw.z);
    }
    for (int e = 0; e < R.T; ++e) {
        const RefTorDev rt = rtor[R.tor_off + e];
        const SideDev sd = side[L.side_off + rt.side];
        const float3 c = lds3(z, sd.c);
        float3 k = sub3(c, lds3(z, sd.b));
        k = mul3(k, rsqrtf(dot3(k, k)));
        float3 s = f3(0.f, 0.f, 0.f);
        for (int j = lane; j < sd.nmov; j += 32) {
            const int i = idx[sd.mov_off + j];
            s = add3(s, cross3(sub3(lds3(z, i), c), lds3(p, i)));
        }
        s = wsum3(s);
        if (lane == 0) put(6 + rt.k, dot3(k, s));
    }
}

#ifdef GEODOCK_CHECKED
// Checked builds: every array a warp of these kernels reads for ligand b lies inside the batch, and every atom
// index it reads lies inside the ligand (codes 1, 2, 3, 4, 8 of GD_OK). Lane 0 checks, the warp agrees.
static __device__ __noinline__ bool ligand_ok(const BatchBounds& B, const LigDev& L, const RefLigDev& R, const SideDev* side,
                                       const uint8_t* idx, const RefTorDev* rtor, int b) {
    bool ok = true;
    if ((threadIdx.x & 31) == 0) {
        unsigned long long* st = B.check;
        ok = GD_OK(st, L.l >= 1 && L.atom_off >= 0 && L.atom_off + L.l <= B.natoms, 1, b) &&
             GD_OK(st, L.l <= B.lmax, 2, b) &&
             GD_OK(st, L.side_off >= 0 && L.side_off + L.nside <= B.nside, 3, b) &&
             GD_OK(st, R.tor_off >= 0 && R.tor_off + R.T <= B.ntor, 8, b) &&
             GD_OK(st, R.check_off >= 0 && R.check_off + L.l * R.wpr <= B.nchk && R.wpr * 32 >= L.l, 8, b);
        for (int e = 0; ok && e < R.T; ++e) {
            const RefTorDev rt = rtor[R.tor_off + e];
            ok = GD_OK(st, rt.side >= 0 && rt.side < L.nside && rt.k >= 0 && rt.k < R.T, 8, b);
            if (!ok) break;
            const SideDev sd = side[L.side_off + rt.side];
            ok = GD_OK(st, sd.mov_off >= 0 && sd.mov_off + sd.nmov <= B.nidx, 3, b) &&
                 GD_OK(st, sd.c < L.l && sd.b < L.l, 4, b);
            for (int j = 0; ok && j < sd.nmov; ++j) ok = GD_OK(st, idx[sd.mov_off + j] < L.l, 4, b);
        }
    }
    return __shfl_sync(FULL, ok ? 1 : 0, 0) != 0;
}
#endif

}  // namespace gd
