// Kernels of the local refinement stage and of the differentiable trilinear
// score (forward and adjoint). The formulas are stated in geodock_refine.cuh.
#include "geodock_refine.cuh"
#include "geodock_refine_launch.h"

namespace gd {

namespace {

// Shared-memory floats per warp.
__host__ __device__ constexpr int refine_warp_floats(int lmax, int tmax) { return 9 * lmax + ((6 + tmax + 3) & ~3); }

// One warp per (pocket, ligand) pair: `steps` ascent steps from xyz_in.
__global__ void __launch_bounds__(128) refine_kernel(RefineParams P, int lmax, int tmax) {
    extern __shared__ float rsm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int pair = blockIdx.x * (blockDim.x >> 5) + warp;
    if (pair >= P.npairs) return;
    float* base = rsm + (size_t)warp * refine_warp_floats(lmax, tmax);
    float* z = base;                 // current pose
    float* zn = base + 3 * lmax;     // trial pose / displacement
    float* p = base + 6 * lmax;      // d o / d z
    float* Gs = base + 9 * lmax;     // d o / d q
    const int pocket = pair / P.nlig, b = pair % P.nlig;
    const LigDev L = P.lig[b];
    const RefLigDev R = P.rlig[b];
#ifdef GEODOCK_CHECKED
    if (!ligand_ok(P.bounds, L, R, P.side, P.idx, P.rtor, b)) return;
#endif
    const PocketDev& pd = P.pockets[pocket];
    const Frame F = frame_of(pd);
    const int l = L.l;
    const bool clip = P.clip != 0;
    const int64_t xo = ((int64_t)pocket * P.natoms + L.atom_off) * 3;
    for (int e = lane; e < 3 * l; e += 32) z[e] = P.xyz_in[xo + e];
    __syncwarp();
    bool inside;
    float S = warp_score(pd, F, z, l, clip, nullptr, &inside);
    const bool skip = clip && !inside;
    if (P.trace_on && lane == 0) {
        P.tr.S_start[pair] = S;
        P.tr.status[pair] = skip ? 1 : 0;
    }
    float lam = REFINE_LAMBDA0;
    const float lf = (float)l;
    for (int st = 0; st < P.steps && !skip; ++st) {
        const int64_t si = (int64_t)pair * P.steps + st;
        // adjoint of o = l / (h^2 S) with respect to the coordinates
        bool dummy;
        warp_score(pd, F, z, l, clip, p, &dummy);
        const float scale = -lf / (F.h2 * S * S);
        __syncwarp();
        for (int e = lane; e < 3 * l; e += 32) p[e] *= scale;
        __syncwarp();
        const float3 g = warp_centroid(z, l);
        const float3 zero = f3(0.f, 0.f, 0.f);
        warp_dof_grad(P.side, P.idx, L, R, P.rtor, z, p, g, zero, zero, [&](int k, float v) { Gs[k] = v; });
        __syncwarp();
        const float3 Gt = f3(Gs[0], Gs[1], Gs[2]), Gw = f3(Gs[3], Gs[4], Gs[5]);
        // largest first-order atom displacement per unit of G
        for (int i = lane; i < l; i += 32) sts3(zn, i, add3(Gt, cross3(Gw, sub3(lds3(z, i), g))));
        __syncwarp();
        for (int e = 0; e < R.T; ++e) {
            const RefTorDev rt = P.rtor[R.tor_off + e];
            const SideDev sd = P.side[L.side_off + rt.side];
            const float3 c = lds3(z, sd.c);
            float3 k = sub3(c, lds3(z, sd.b));
            k = mul3(k, rsqrtf(dot3(k, k)));
            const float gk = Gs[6 + rt.k];
            for (int j = lane; j < sd.nmov; j += 32) {
                const int i = P.idx[sd.mov_off + j];
                sts3(zn, i, add3(lds3(zn, i), mul3(cross3(k, sub3(lds3(z, i), c)), gk)));
            }
            __syncwarp();
        }
        float D = 0.f;
        for (int i = lane; i < l; i += 32) {
            const float3 d = lds3(zn, i);
            D = fmaxf(D, sqrtf(dot3(d, d)));
        }
        D = wmax(D);
        if (P.trace_on && lane == 0) {
            for (int k = 0; k < 6 + R.T; ++k) P.tr.G[si * P.tr.gstride + k] = Gs[k];
            P.tr.D[si] = D;
            P.tr.lam[si] = lam;
        }
        int verdict = 0;
        float S_new = S;
        if (D > 0.f) {
            const float f = lam / D;
            __syncwarp();
            for (int e = lane; e < 3 * l; e += 32) zn[e] = z[e];
            __syncwarp();
            warp_torsions(P.side, P.idx, L, R, P.rtor, zn, [&](int k) { return Gs[6 + k] * f; });
            warp_rigid(zn, l, g, mul3(Gt, f), mul3(Gw, f));
            bool in_new;
            S_new = warp_score(pd, F, zn, l, clip, nullptr, &in_new);
            // bump check over every pair a torsion moves
            bool clash = false;
            for (int i = lane; i < l; i += 32) {
                const uint32_t* row = P.check + R.check_off + (int64_t)i * R.wpr;
                const float3 zi = lds3(zn, i);
                for (int w = 0; w < R.wpr; ++w) {
                    uint32_t bits = row[w];
                    const int lo = i - 32 * w;  // keep j > i only
                    if (lo >= 31) bits = 0u;
                    else if (lo >= 0) bits &= ~((2u << lo) - 1u);
                    while (bits) {
                        const int j = 32 * w + __ffs(bits) - 1;
                        bits &= bits - 1u;
                        const float3 d = sub3(zi, lds3(zn, j));
                        if (dot3(d, d) < P.thr2) clash = true;
                    }
                }
            }
            clash = __any_sync(FULL, clash);
            verdict = (S_new < S ? 1 : 0) | (clash ? 0 : 2) | (in_new ? 4 : 0);
        }
        const bool acc = (verdict & 1) && (verdict & 2) && (!clip || (verdict & 4));
        if (P.trace_on && lane == 0) {
            P.tr.S_new[si] = S_new;
            P.tr.verdict[si] = verdict;
            P.tr.accept[si] = acc ? 1 : 0;
        }
        if (acc) {
            float* t = z;
            z = zn;
            zn = t;
            S = S_new;
            lam = fminf(lam * REFINE_GROW, REFINE_LAMBDA_MAX);
        } else {
            lam *= REFINE_SHRINK;
        }
        __syncwarp();
    }
    for (int e = lane; e < 3 * l; e += 32) P.xyz_out[xo + e] = z[e];
    if (lane == 0) {
        if (P.trace_on) P.tr.S_final[pair] = S;
        int32_t* w = reinterpret_cast<int32_t*>(P.result + (int64_t)pair * 4);
        P.result[(int64_t)pair * 4] = skip ? 0.f : (float)((double)l / (pd.h * pd.h * (double)S));
        w[1] = -1;
        w[2] = skip ? 1 : 0;
        w[3] = 0;
    }
}

// o = l / (h^2 S) per ligand.
__global__ void __launch_bounds__(128) score_fwd_kernel(ScoreParams P, int lmax) {
    extern __shared__ float rsm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int b = blockIdx.x * (blockDim.x >> 5) + warp;
    if (b >= P.nlig) return;
    float* z = rsm + (size_t)warp * 3 * lmax;
    const LigDev L = P.lig[b];
#ifdef GEODOCK_CHECKED
    if (!ligand_ok(P.bounds, L, P.rlig[b], P.side, P.idx, P.rtor, b)) return;
#endif
    const PocketDev& pd = *P.pocket;
    for (int e = lane; e < 3 * L.l; e += 32) z[e] = P.x[(int64_t)L.atom_off * 3 + e];
    __syncwarp();
    bool in;
    const float S = warp_score(pd, frame_of(pd), z, L.l, P.clip != 0, nullptr, &in);
    if (lane == 0) P.out[b] = (float)((double)L.l / (pd.h * pd.h * (double)S));
}

// d L / d x_i = (d L / d o) (-l / (h^2 S^2)) d S / d x_i.
__global__ void __launch_bounds__(128) score_bwd_kernel(ScoreParams P, int lmax) {
    extern __shared__ float rsm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int b = blockIdx.x * (blockDim.x >> 5) + warp;
    if (b >= P.nlig) return;
    float* z = rsm + (size_t)warp * 6 * lmax;
    float* dS = z + 3 * lmax;
    const LigDev L = P.lig[b];
#ifdef GEODOCK_CHECKED
    if (!ligand_ok(P.bounds, L, P.rlig[b], P.side, P.idx, P.rtor, b)) return;
#endif
    const PocketDev& pd = *P.pocket;
    const Frame F = frame_of(pd);
    for (int e = lane; e < 3 * L.l; e += 32) z[e] = P.x[(int64_t)L.atom_off * 3 + e];
    __syncwarp();
    bool in;
    const float S = warp_score(pd, F, z, L.l, P.clip != 0, dS, &in);
    const float go = P.grad_in ? P.grad_in[b] : 1.f;
    const float scale = go * (-(float)L.l / (F.h2 * S * S));
    __syncwarp();
    for (int e = lane; e < 3 * L.l; e += 32) P.out[(int64_t)L.atom_off * 3 + e] = dS[e] * scale;
}

// z = apply(x, q) into the warp's buffer y (shared memory); returns the centroid of x.
__device__ __forceinline__ float3 apply_dofs(const ScoreParams& P, const LigDev& L, const RefLigDev& R, int b, float* y) {
    const int lane = threadIdx.x & 31;
    for (int e = lane; e < 3 * L.l; e += 32) y[e] = P.x[(int64_t)L.atom_off * 3 + e];
    __syncwarp();
    const float3 g = warp_centroid(y, L.l);
    const float* q = P.q + (int64_t)b * P.qstride;
    warp_torsions(P.side, P.idx, L, R, P.rtor, y, [&](int k) { return q[6 + k]; });
    warp_rigid(y, L.l, g, f3(q[0], q[1], q[2]), f3(q[3], q[4], q[5]));
    return g;
}

__global__ void __launch_bounds__(128) dof_apply_kernel(ScoreParams P, int lmax) {
    extern __shared__ float rsm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int b = blockIdx.x * (blockDim.x >> 5) + warp;
    if (b >= P.nlig) return;
    float* y = rsm + (size_t)warp * 3 * lmax;
    const LigDev L = P.lig[b];
    const RefLigDev R = P.rlig[b];
#ifdef GEODOCK_CHECKED
    if (!ligand_ok(P.bounds, L, R, P.side, P.idx, P.rtor, b)) return;
#endif
    apply_dofs(P, L, R, b, y);
    for (int e = lane; e < 3 * L.l; e += 32) P.out[(int64_t)L.atom_off * 3 + e] = y[e];
}

// d L / d q = J(q)^T d L / d z.
__global__ void __launch_bounds__(128) dof_grad_kernel(ScoreParams P, int lmax) {
    extern __shared__ float rsm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int b = blockIdx.x * (blockDim.x >> 5) + warp;
    if (b >= P.nlig) return;
    float* y = rsm + (size_t)warp * 6 * lmax;
    float* p = y + 3 * lmax;
    const LigDev L = P.lig[b];
    const RefLigDev R = P.rlig[b];
#ifdef GEODOCK_CHECKED
    if (!ligand_ok(P.bounds, L, R, P.side, P.idx, P.rtor, b)) return;
#endif
    const float3 g = apply_dofs(P, L, R, b, y);
    for (int e = lane; e < 3 * L.l; e += 32) p[e] = P.grad_in[(int64_t)L.atom_off * 3 + e];
    __syncwarp();
    const float* q = P.q + (int64_t)b * P.qstride;
    float* G = P.out + (int64_t)b * P.qstride;
    for (int k = 6 + R.T + lane; k < P.qstride; k += 32) G[k] = 0.f;
    warp_dof_grad(P.side, P.idx, L, R, P.rtor, y, p, g, f3(q[0], q[1], q[2]), f3(q[3], q[4], q[5]),
                  [&](int k, float v) { G[k] = v; });
}

constexpr int WARPS = 4;

cudaError_t smem_attr(const void* fn, size_t smem) {
    if (smem <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

}  // namespace

cudaError_t launch_refine(const RefineParams& P, int lmax, int tmax, cudaStream_t s) {
    if (P.npairs == 0) return cudaSuccess;
    const size_t smem = (size_t)WARPS * refine_warp_floats(lmax, tmax) * sizeof(float);
    cudaError_t e = smem_attr((const void*)refine_kernel, smem);
    if (e != cudaSuccess) return e;
    refine_kernel<<<(P.npairs + WARPS - 1) / WARPS, 32 * WARPS, smem, s>>>(P, lmax, tmax);
    return cudaGetLastError();
}

cudaError_t launch_score(const ScoreParams& P, int lmax, int which, cudaStream_t s) {
    if (P.nlig == 0) return cudaSuccess;
    const int grid = (P.nlig + WARPS - 1) / WARPS;
    const size_t one = (size_t)WARPS * 3 * lmax * sizeof(float);
    cudaError_t e = cudaSuccess;
    switch (which) {
        case SCORE_FWD:
            e = smem_attr((const void*)score_fwd_kernel, one);
            if (e == cudaSuccess) score_fwd_kernel<<<grid, 32 * WARPS, one, s>>>(P, lmax);
            break;
        case SCORE_BWD:
            e = smem_attr((const void*)score_bwd_kernel, 2 * one);
            if (e == cudaSuccess) score_bwd_kernel<<<grid, 32 * WARPS, 2 * one, s>>>(P, lmax);
            break;
        case DOF_APPLY:
            e = smem_attr((const void*)dof_apply_kernel, one);
            if (e == cudaSuccess) dof_apply_kernel<<<grid, 32 * WARPS, one, s>>>(P, lmax);
            break;
        case DOF_GRAD:
            e = smem_attr((const void*)dof_grad_kernel, 2 * one);
            if (e == cudaSuccess) dof_grad_kernel<<<grid, 32 * WARPS, 2 * one, s>>>(P, lmax);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace gd
