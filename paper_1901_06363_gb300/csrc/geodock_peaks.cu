// Rates that bound the sweep kernel, measured on the device it runs on
// (measurement only; nothing on the docking path calls these):
//   - FP32 fused multiply-adds per second: scalar fmaf and packed __ffma2_rn
//     (two per instruction), eight independent chains per thread;
//   - point-sampled fetches per second from a pocket's padded-field texture:
//     spread over the whole field (L2-resident), and confined to a 16^3-voxel
//     cube per warp (L1-resident, the locality of one ligand's poses);
//   - random 32-byte sector loads per second from a 64 MiB buffer held in L2.
// Each is timed with CUDA events on the given stream after one warm-up launch.
#include <cuda_runtime.h>

#include <cstdint>

#include "geodock_launch.h"

namespace gd {

namespace {

constexpr int CHAINS = 8;

__global__ void fma_rate_kernel(float* out, int iters, float a, float b) {
    float x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = (float)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) x[c] = __fmaf_rn(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void ffma2_rate_kernel(float* out, int iters, float a, float b) {
    float2 x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = make_float2((float)(threadIdx.x + c), (float)c);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c].x + x[c].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Coordinates walk by fixed strides with wrap-around inside [0, ext) (whole
// field) or inside a 16-voxel cube at a per-warp corner (local).
__global__ void tex_rate_kernel(unsigned long long tex, unsigned* out, int iters, float ex, float ey, float ez,
                                int local) {
    const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned warp = tid >> 5;
    unsigned h = tid * 2654435761u + 12345u;
    float span_x = ex, span_y = ey, span_z = ez, ox = 0.f, oy = 0.f, oz = 0.f;
    if (local) {
        span_x = span_y = span_z = 16.f;
        unsigned w = warp * 2246822519u + 7u;
        ox = (float)(w % (unsigned)(ex - 16.f));
        w = w * 3266489917u + 11u;
        oy = (float)(w % (unsigned)(ey - 16.f));
        w = w * 668265263u + 13u;
        oz = (float)(w % (unsigned)(ez - 16.f));
    }
    float x = (float)(h % 1000u) * 1e-3f * span_x;
    h = h * 1103515245u + 12345u;
    float y = (float)(h % 1000u) * 1e-3f * span_y;
    h = h * 1103515245u + 12345u;
    float z = (float)(h % 1000u) * 1e-3f * span_z;
    unsigned acc = 0;
    for (int i = 0; i < iters; ++i) {
        acc += tex3D<unsigned>(tex, ox + x, oy + y, oz + z);
        x += 5.37f;
        y += 3.11f;
        z += 2.29f;
        x = x >= span_x ? x - span_x : x;
        y = y >= span_y ? y - span_y : y;
        z = z >= span_z ? z - span_z : z;
    }
    out[tid] = acc;
}

__global__ void l2_rate_kernel(const unsigned* __restrict__ buf, unsigned nwords, unsigned* out, int iters) {
    const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned h = tid * 2654435761u + 1u;
    unsigned acc = 0;
    const unsigned nsect = nwords / 8u;  // 32-byte sectors
    for (int i = 0; i < iters; ++i) {
        h = h * 1664525u + 1013904223u;
        acc += __ldcg(buf + (size_t)(h % nsect) * 8u);
    }
    out[tid] = acc;
}

__global__ void fill_kernel(unsigned* buf, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        buf[i] = (unsigned)i;
}

template <class F>
cudaError_t time_ms(cudaStream_t s, F launch, float* ms) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = launch();  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return e;
}

}  // namespace

cudaError_t measure_peaks(unsigned long long tex, int px, int py, int pz, int num_sms, cudaStream_t s, double* r) {
    const int block = 256, grid = num_sms * 8;  // 2,048 threads per SM
    const size_t threads = (size_t)grid * block;
    unsigned* out = nullptr;
    unsigned* buf = nullptr;
    const size_t nwords = (size_t)64 << 18;  // 64 MiB
    cudaError_t e = cudaMalloc(&out, threads * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&buf, nwords * sizeof(unsigned));
    float ms = 0.f;
    // FP32 FMA, scalar and packed
    const int fiters = 32768;
    if (e == cudaSuccess)
        e = time_ms(s, [&]() {
            fma_rate_kernel<<<grid, block, 0, s>>>(reinterpret_cast<float*>(out), fiters, 0.999f, 1e-3f);
            return cudaGetLastError();
        }, &ms);
    if (e == cudaSuccess) r[0] = (double)threads * fiters * CHAINS / (ms * 1e-3);
    if (e == cudaSuccess)
        e = time_ms(s, [&]() {
            ffma2_rate_kernel<<<grid, block, 0, s>>>(reinterpret_cast<float*>(out), fiters, 0.999f, 1e-3f);
            return cudaGetLastError();
        }, &ms);
    if (e == cudaSuccess) r[1] = (double)threads * fiters * CHAINS * 2 / (ms * 1e-3);
    // texture fetches over the field, then within 16^3 cubes
    const int titers = 8192;
    for (int local = 0; local < 2 && e == cudaSuccess; ++local) {
        e = time_ms(s, [&]() {
            tex_rate_kernel<<<grid, block, 0, s>>>(tex, out, titers, (float)px, (float)py, (float)pz, local);
            return cudaGetLastError();
        }, &ms);
        if (e == cudaSuccess) r[2 + local] = (double)threads * titers / (ms * 1e-3);
    }
    // random 32-byte sectors from an L2-resident buffer (filled first, so it is resident)
    const int liters = 4096;
    if (e == cudaSuccess) {
        fill_kernel<<<grid, block, 0, s>>>(buf, nwords);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = time_ms(s, [&]() {
            l2_rate_kernel<<<grid, block, 0, s>>>(buf, (unsigned)nwords, out, liters);
            return cudaGetLastError();
        }, &ms);
    if (e == cudaSuccess) r[4] = (double)threads * liters / (ms * 1e-3);
    if (out) cudaFree(out);
    if (buf) cudaFree(buf);
    return e;
}

}  // namespace gd
