// nbody.cu -- the consumer: one all-pairs n-body step through a view.
//
// The paper's Fig. 2 shows the update loop (for each i, interact with every
// j, then store the velocity) and Sec. 5 names the move phase.  Here:
//   update: v_i += dt * sum_j m_j d_ij / (|d_ij|^2 + eps^2)^(3/2), d_ij = p_j - p_i
//   move:   p_i += dt * v_i
// Particles are read and written through the view's mapping (AoS, SoA single
// or multi blob, AoSoA with a power-of-two lane count); the arithmetic does not
// depend on the mapping, so every mapping gives the same bits.
//
// Each block owns kI particles and splits the j range into kParts equal
// slices, one warp each; a slice streams kJ-particle tiles through shared
// memory.  The tile is a view with compile-time extents (Sec. 2: stateless
// extents make a view storage-equivalent to its data, so it can live in
// shared memory): it holds nothing but the {x, y, z, m} records.  Per-slice
// partial sums are added in a fixed order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"

namespace llgb {

// Compile-time specialisations of the address function for the common
// mappings; PV_GENERIC reads the runtime parameters.
template <int KIND>
struct Addr {
    __device__ __forceinline__ static uint64_t off(const ParticleView& v, uint32_t i)
    {
        if (KIND == PV_AOS) return (uint64_t)i * 28u;
        if (KIND == PV_SOA) return (uint64_t)i * 4u;
        if (KIND == PV_AOSOA32) return (uint64_t)(i >> 5) * (32u * 28u) + (i & 31u) * 4u;
        return (uint64_t)(i >> v.lshift) * v.bstride + (uint64_t)(i & v.lmask) * 4u;
    }
};

template <int KIND>
__device__ __forceinline__ float ld_leaf(const ParticleView& v, int f, uint32_t i)
{
    return *reinterpret_cast<const float*>(v.base[f] + Addr<KIND>::off(v, i));
}

template <int KIND>
__device__ __forceinline__ void st_leaf(const ParticleView& v, int f, uint32_t i, float x)
{
    *reinterpret_cast<float*>(v.base[f] + Addr<KIND>::off(v, i)) = x;
}

// A shared-memory view with compile-time extent N of the record {x, y, z, m}:
// no extents or mapping state are stored, only the records.
template <int N>
struct StaticBodyTile {
    float4 rec[N];
    __device__ __forceinline__ float4& operator()(int j) { return rec[j]; }
};

constexpr int kW = 32;              // threads per j slice: one warp
constexpr int kIPT = 2;             // particles per thread (two chains per j record)
constexpr int kI = kW * kIPT;       // particles per block
constexpr int kParts = 8;           // j slices per block, one per warp
constexpr int kJ = 128;             // tile extent (4 records per loading lane)

// Interaction of particle p with record b = {x, y, z, m}, summed into t.
__device__ __forceinline__ void interact(const float4 b, float px, float py, float pz, float eps2, float& tx,
                                         float& ty, float& tz)
{
    const float dx = b.x - px, dy = b.y - py, dz = b.z - pz;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
    const float rinv = rsqrtf(r2);
    const float s = b.w * (rinv * rinv * rinv);
    tx = fmaf(dx, s, tx);
    ty = fmaf(dy, s, ty);
    tz = fmaf(dz, s, tz);
}

// One warp per j slice: it stages kJ-record tiles of its slice with warp-
// level synchronisation only, and every lane interacts two particles (i and
// i + 32) with each staged record.
template <int KIND>
__global__ void __launch_bounds__(kW * kParts) nbody_update(const ParticleView v, float eps2, float dt,
                                                            uint32_t chunk)
{
    __shared__ StaticBodyTile<kJ> tile[kParts];
    __shared__ float3 partial[kParts][kI];
    const uint32_t lane = threadIdx.x % kW;
    const uint32_t part = threadIdx.x / kW;
    const uint32_t i0 = blockIdx.x * kI + lane, i1 = i0 + kW;
    const uint32_t n = v.n;

    float p0x = 0.f, p0y = 0.f, p0z = 0.f, p1x = 0.f, p1y = 0.f, p1z = 0.f;
    if (i0 < n) {
        p0x = ld_leaf<KIND>(v, 0, i0);
        p0y = ld_leaf<KIND>(v, 1, i0);
        p0z = ld_leaf<KIND>(v, 2, i0);
    }
    if (i1 < n) {
        p1x = ld_leaf<KIND>(v, 0, i1);
        p1y = ld_leaf<KIND>(v, 1, i1);
        p1z = ld_leaf<KIND>(v, 2, i1);
    }
    float a0x = 0.f, a0y = 0.f, a0z = 0.f, a1x = 0.f, a1y = 0.f, a1z = 0.f;
    const uint32_t j0 = part * chunk;
    for (uint32_t jt = 0; jt < chunk; jt += kJ) {
#pragma unroll
        for (int r = 0; r < kJ / kW; ++r) {
            const uint32_t jl = jt + lane + r * kW;
            const uint32_t j = j0 + jl;
            float4 q = make_float4(0.f, 0.f, 0.f, 0.f);  // zero mass beyond n
            if (j < n && jl < chunk)
                q = make_float4(ld_leaf<KIND>(v, 0, j), ld_leaf<KIND>(v, 1, j), ld_leaf<KIND>(v, 2, j),
                                ld_leaf<KIND>(v, 6, j));
            tile[part](lane + r * kW) = q;
        }
        __syncwarp();
        float t0x = 0.f, t0y = 0.f, t0z = 0.f, t1x = 0.f, t1y = 0.f, t1z = 0.f;
#pragma unroll 8
        for (int jj = 0; jj < kJ; ++jj) {
            const float4 b = tile[part](jj);
            interact(b, p0x, p0y, p0z, eps2, t0x, t0y, t0z);
            interact(b, p1x, p1y, p1z, eps2, t1x, t1y, t1z);
        }
        a0x += t0x;
        a0y += t0y;
        a0z += t0z;
        a1x += t1x;
        a1y += t1y;
        a1z += t1z;
        __syncwarp();
    }
    partial[part][lane] = make_float3(a0x, a0y, a0z);
    partial[part][lane + kW] = make_float3(a1x, a1y, a1z);
    __syncthreads();
    // warp 0 adds the slices in a fixed order, one particle per lane and pass
    if (part == 0) {
#pragma unroll
        for (int h = 0; h < kIPT; ++h) {
            const uint32_t li = lane + h * kW;
            const uint32_t i = blockIdx.x * kI + li;
            if (i >= n) continue;
            float sx = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll
            for (int p = 0; p < kParts; ++p) {
                sx += partial[p][li].x;
                sy += partial[p][li].y;
                sz += partial[p][li].z;
            }
            st_leaf<KIND>(v, 3, i, fmaf(dt, sx, ld_leaf<KIND>(v, 3, i)));
            st_leaf<KIND>(v, 4, i, fmaf(dt, sy, ld_leaf<KIND>(v, 4, i)));
            st_leaf<KIND>(v, 5, i, fmaf(dt, sz, ld_leaf<KIND>(v, 5, i)));
        }
    }
}

template <int KIND>
__global__ void nbody_move(const ParticleView v, float dt)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.n) return;
    for (int k = 0; k < 3; ++k) st_leaf<KIND>(v, k, i, fmaf(dt, ld_leaf<KIND>(v, 3 + k, i), ld_leaf<KIND>(v, k, i)));
}

template <int KIND>
static cudaError_t launch_kind(const ParticleView& v, float eps, float dt, cudaStream_t stream)
{
    const uint32_t n = v.n;
    uint32_t chunk = (n + kParts - 1) / kParts;
    chunk = (chunk + kJ - 1) / kJ * kJ;
    const uint32_t blocks = (n + kI - 1) / kI;
    nbody_update<KIND><<<blocks, kW * kParts, 0, stream>>>(v, eps * eps, dt, chunk);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    nbody_move<KIND><<<(n + 255) / 256, 256, 0, stream>>>(v, dt);
    return cudaGetLastError();
}

cudaError_t launch_nbody(const ParticleView& v, int kind, float eps, float dt, cudaStream_t stream)
{
    if (v.n == 0) return cudaSuccess;
    switch (kind) {
    case PV_AOS: return launch_kind<PV_AOS>(v, eps, dt, stream);
    case PV_SOA: return launch_kind<PV_SOA>(v, eps, dt, stream);
    case PV_AOSOA32: return launch_kind<PV_AOSOA32>(v, eps, dt, stream);
    default: return launch_kind<PV_GENERIC>(v, eps, dt, stream);
    }
}

}  // namespace llgb
