// nbody.cu -- tier 1 of the recommendation tool (Sec. 2) on this GPU: a direct (all-pairs)
// n-body code, NB of Sec. 3.2, whose six source-code optimizations of Sec. 3.3 are compile-time
// switches, so that one binary holds all 64 versions (one template instantiation per 6-bit
// optimization mask).  Bits (the order the speedup-prediction path uses for this code):
//   0 CONST   immutable kernel parameters read from constant memory, not passed per launch
//   1 PEEL    the innermost loop split into a loop over whole chunks of a compile-time count
//             and a remainder loop
//   2 SHMEM   the bodies staged through shared memory in block-sized tiles (blocking)
//   3 UNROLL  the innermost loop unrolled (a pragma) instead of kept rolled
//   4 FTZ     single-precision arithmetic that flushes denormals to zero (the .ftz forms)
//   5 RSQRT   the reciprocal square root intrinsic instead of 1 / sqrt
// Each time step computes every body's acceleration from all bodies (softened gravity) and
// advances velocities and positions (semi-implicit Euler).
//
// Usage: nbody time <bodies> <steps> <reps>    per version: median time of a run of <steps>
//                                              time steps over <reps> runs (CUDA events), CSV
//        nbody run <mask> <bodies> <steps>     one run of one version
//        nbody profile <mask> <bodies>...      one time step of one version per body count
//                                              (the launches a profiler captures)
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <utility>
#include <vector>

namespace {

struct Params {
    const float4* pos_in;    // x, y, z, mass
    float4* pos_out;
    float4* vel;             // vx, vy, vz, unused
    int n;
    float dt;
    float eps2;
};

__constant__ Params c_par;

constexpr int kBlock = 256;
constexpr int kChunk = 32;

template <bool FTZ>
__device__ __forceinline__ float fadd(float a, float b) {
    if constexpr (FTZ) {
        float r;
        asm("add.ftz.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
        return r;
    } else {
        return __fadd_rn(a, b);
    }
}
template <bool FTZ>
__device__ __forceinline__ float fmul(float a, float b) {
    if constexpr (FTZ) {
        float r;
        asm("mul.ftz.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
        return r;
    } else {
        return __fmul_rn(a, b);
    }
}
template <bool FTZ>
__device__ __forceinline__ float ffma(float a, float b, float c) {
    if constexpr (FTZ) {
        float r;
        asm("fma.rn.ftz.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
        return r;
    } else {
        return __fmaf_rn(a, b, c);
    }
}
template <bool FTZ, bool RSQRT>
__device__ __forceinline__ float inv_sqrt(float x) {
    if constexpr (RSQRT) {
        if constexpr (FTZ) {
            float r;
            asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
            return r;
        } else {
            return rsqrtf(x);
        }
    } else {
        if constexpr (FTZ) {
            float s, r;
            asm("sqrt.rn.ftz.f32 %0, %1;" : "=f"(s) : "f"(x));
            asm("div.rn.ftz.f32 %0, %1, %2;" : "=f"(r) : "f"(1.0f), "f"(s));
            return r;
        } else {
            return 1.0f / sqrtf(x);
        }
    }
}

// acceleration on a body at p from body q (softened): a += m_q d / (|d|^2 + eps^2)^(3/2)
template <bool FTZ, bool RSQRT>
__device__ __forceinline__ void interact(const float4& p, const float4& q, float eps2, float3& a) {
    const float dx = fadd<FTZ>(q.x, -p.x), dy = fadd<FTZ>(q.y, -p.y), dz = fadd<FTZ>(q.z, -p.z);
    const float d2 = ffma<FTZ>(dx, dx, ffma<FTZ>(dy, dy, ffma<FTZ>(dz, dz, eps2)));
    const float inv = inv_sqrt<FTZ, RSQRT>(d2);
    const float s = fmul<FTZ>(q.w, fmul<FTZ>(inv, fmul<FTZ>(inv, inv)));
    a.x = ffma<FTZ>(dx, s, a.x);
    a.y = ffma<FTZ>(dy, s, a.y);
    a.z = ffma<FTZ>(dz, s, a.z);
}

template <bool FTZ, bool RSQRT, bool UNROLL>
__device__ __forceinline__ void span(const float4& p, const float4* src, int cnt, float eps2, float3& a) {
    if constexpr (UNROLL) {
#pragma unroll 8
        for (int j = 0; j < cnt; ++j) interact<FTZ, RSQRT>(p, src[j], eps2, a);
    } else {
#pragma unroll 1
        for (int j = 0; j < cnt; ++j) interact<FTZ, RSQRT>(p, src[j], eps2, a);
    }
}

// bodies [0, cnt) of src: with PEEL a loop over whole chunks of kChunk, then the remainder
template <bool FTZ, bool RSQRT, bool UNROLL, bool PEEL>
__device__ __forceinline__ void all_of(const float4& p, const float4* src, int cnt, float eps2, float3& a) {
    if constexpr (PEEL) {
        const int whole = cnt - cnt % kChunk;
        for (int j0 = 0; j0 < whole; j0 += kChunk) {
            if constexpr (UNROLL) {
#pragma unroll
                for (int j = 0; j < kChunk; ++j) interact<FTZ, RSQRT>(p, src[j0 + j], eps2, a);
            } else {
#pragma unroll 1
                for (int j = 0; j < kChunk; ++j) interact<FTZ, RSQRT>(p, src[j0 + j], eps2, a);
            }
        }
        span<FTZ, RSQRT, UNROLL>(p, src + whole, cnt - whole, eps2, a);
    } else {
        span<FTZ, RSQRT, UNROLL>(p, src, cnt, eps2, a);
    }
}

template <int MASK>
__global__ void __launch_bounds__(kBlock) nbody_step(Params arg) {
    constexpr bool CONST = MASK & 1, PEEL = MASK & 2, SHMEM = MASK & 4, UNROLL = MASK & 8, FTZ = MASK & 16,
                   RSQRT = MASK & 32;
    const Params& P = CONST ? c_par : arg;
    const int i = blockIdx.x * kBlock + threadIdx.x;
    const int n = P.n;
    const float4 p = i < n ? P.pos_in[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    float3 a = make_float3(0.f, 0.f, 0.f);
    if constexpr (SHMEM) {
        __shared__ float4 tile[kBlock];
        for (int t0 = 0; t0 < n; t0 += kBlock) {
            const int j = t0 + threadIdx.x;
            tile[threadIdx.x] = j < n ? P.pos_in[j] : make_float4(0.f, 0.f, 0.f, 0.f);
            __syncthreads();
            const int cnt = n - t0 < kBlock ? n - t0 : kBlock;
            all_of<FTZ, RSQRT, UNROLL, PEEL>(p, tile, cnt, P.eps2, a);
            __syncthreads();
        }
    } else {
        all_of<FTZ, RSQRT, UNROLL, PEEL>(p, P.pos_in, n, P.eps2, a);
    }
    if (i < n) {
        float4 v = P.vel[i];
        v.x = ffma<FTZ>(a.x, P.dt, v.x);
        v.y = ffma<FTZ>(a.y, P.dt, v.y);
        v.z = ffma<FTZ>(a.z, P.dt, v.z);
        P.vel[i] = v;
        P.pos_out[i] = make_float4(ffma<FTZ>(v.x, P.dt, p.x), ffma<FTZ>(v.y, P.dt, p.y),
                                   ffma<FTZ>(v.z, P.dt, p.z), p.w);
    }
}

using Kern = void (*)(Params);
template <int... M>
constexpr auto table(std::integer_sequence<int, M...>) {
    return std::array<Kern, sizeof...(M)>{nbody_step<M>...};
}
const auto kKernels = table(std::make_integer_sequence<int, 64>{});

#define CK(x)                                                                          \
    do {                                                                               \
        cudaError_t e_ = (x);                                                          \
        if (e_ != cudaSuccess) {                                                       \
            fprintf(stderr, "%s:%d %s\n", __FILE__, __LINE__, cudaGetErrorString(e_)); \
            exit(1);                                                                   \
        }                                                                              \
    } while (0)

struct Sim {
    int n;
    float4 *pos[2], *vel;
    std::vector<float4> p0, v0;
    explicit Sim(int n_) : n(n_) {
        CK(cudaMalloc(&pos[0], n * sizeof(float4)));
        CK(cudaMalloc(&pos[1], n * sizeof(float4)));
        CK(cudaMalloc(&vel, n * sizeof(float4)));
        // a Plummer-like cloud from a fixed linear congruential stream (the same bodies for
        // every version and run)
        p0.resize(n);
        v0.resize(n);
        unsigned long long s = 0x9E3779B97F4A7C15ull ^ (unsigned long long)n;
        auto u = [&]() {
            s = s * 6364136223846793005ull + 1442695040888963407ull;
            return (float)((s >> 40) & 0xFFFFFF) / 16777216.0f;
        };
        for (int i = 0; i < n; ++i) {
            const float r = 1.0f / sqrtf(powf(u() * 0.999f + 1e-3f, -2.0f / 3.0f) - 1.0f + 1e-6f);
            const float ct = 2.0f * u() - 1.0f, ph = 6.2831853f * u(), st = sqrtf(1.0f - ct * ct);
            p0[i] = make_float4(r * st * cosf(ph), r * st * sinf(ph), r * ct, 1.0f / n);
            v0[i] = make_float4(0.1f * (u() - 0.5f), 0.1f * (u() - 0.5f), 0.1f * (u() - 0.5f), 0.f);
        }
    }
    ~Sim() {
        cudaFree(pos[0]);
        cudaFree(pos[1]);
        cudaFree(vel);
    }
    void reset() {
        CK(cudaMemcpy(pos[0], p0.data(), n * sizeof(float4), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(vel, v0.data(), n * sizeof(float4), cudaMemcpyHostToDevice));
    }
    // steps time steps of version mask; returns the GPU time in ms
    float run(int mask, int steps) {
        reset();
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        const int blocks = (n + kBlock - 1) / kBlock;
        CK(cudaEventRecord(e0));
        for (int t = 0; t < steps; ++t) {
            Params P{pos[t & 1], pos[(t + 1) & 1], vel, n, 1e-3f, 1e-4f};
            if (mask & 1) CK(cudaMemcpyToSymbolAsync(c_par, &P, sizeof(P)));
            kKernels[mask]<<<blocks, kBlock>>>(P);
            CK(cudaGetLastError());
        }
        CK(cudaEventRecord(e1));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return ms;
    }
};

}  // namespace

int main(int argc, char** argv) {
    if (argc >= 5 && !strcmp(argv[1], "time")) {
        const int n = atoi(argv[2]), steps = atoi(argv[3]), reps = atoi(argv[4]);
        if (n < 1 || n > (1 << 22) || steps < 1 || reps < 1) return 2;
        Sim sim(n);
        sim.run(0, 1);                                   // warm-up
        printf("mask,bodies,steps,ms_median\n");
        for (int mask = 0; mask < 64; ++mask) {
            std::vector<float> t;
            for (int r = 0; r < reps; ++r) t.push_back(sim.run(mask, steps));
            std::sort(t.begin(), t.end());
            printf("%d,%d,%d,%.6f\n", mask, n, steps, t[t.size() / 2]);
        }
        return 0;
    }
    if (argc >= 5 && !strcmp(argv[1], "run")) {
        const int mask = atoi(argv[2]), n = atoi(argv[3]), steps = atoi(argv[4]);
        if (mask < 0 || mask > 63 || n < 1 || n > (1 << 22) || steps < 1) return 2;
        Sim sim(n);
        printf("%.6f\n", sim.run(mask, steps));
        return 0;
    }
    if (argc >= 4 && !strcmp(argv[1], "profile")) {
        const int mask = atoi(argv[2]);
        if (mask < 0 || mask > 63) return 2;
        for (int a = 3; a < argc; ++a) {
            const int n = atoi(argv[a]);
            if (n < 1 || n > (1 << 22)) return 2;
            Sim sim(n);
            sim.run(mask, 1);
        }
        return 0;
    }
    fprintf(stderr, "usage: nbody time <bodies> <steps> <reps> | nbody run <mask> <bodies> <steps> | "
                    "nbody profile <mask> <bodies>...\n");
    return 2;
}
