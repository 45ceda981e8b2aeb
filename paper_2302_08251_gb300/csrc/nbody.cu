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
// slices; every slice streams kJ-particle tiles through shared memory.  The
// tile is a view with compile-time extents (Sec. 2: stateless extents make a
// view storage-equivalent to its data, so it can live in shared memory): it
// holds nothing but the {x, y, z, m} records.  Per-slice partial sums are
// added in a fixed order.
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

constexpr int kI = 64;      // particles per block
constexpr int kParts = 4;   // j slices per particle
constexpr int kJ = 64;      // tile extent (one record per loading thread)
static_assert(kJ == kI, "each thread of a slice loads one tile record");

template <int KIND>
__global__ void __launch_bounds__(kI * kParts) nbody_update(const ParticleView v, float eps2, float dt,
                                                            uint32_t chunk)
{
    __shared__ StaticBodyTile<kJ> tile[kParts];
    __shared__ float3 partial[kParts][kI];
    const uint32_t li = threadIdx.x % kI;
    const uint32_t part = threadIdx.x / kI;
    const uint32_t i = blockIdx.x * kI + li;
    const uint32_t n = v.n;

    float px = 0.f, py = 0.f, pz = 0.f;
    if (i < n) {
        px = ld_leaf<KIND>(v, 0, i);
        py = ld_leaf<KIND>(v, 1, i);
        pz = ld_leaf<KIND>(v, 2, i);
    }
    float ax = 0.f, ay = 0.f, az = 0.f;
    const uint32_t j0 = part * chunk;
    for (uint32_t jt = 0; jt < chunk; jt += kJ) {
        const uint32_t j = j0 + jt + li;
        float4 q = make_float4(0.f, 0.f, 0.f, 0.f);  // zero mass beyond n
        if (j < n && jt + li < chunk)
            q = make_float4(ld_leaf<KIND>(v, 0, j), ld_leaf<KIND>(v, 1, j), ld_leaf<KIND>(v, 2, j),
                            ld_leaf<KIND>(v, 6, j));
        tile[part](li) = q;
        __syncthreads();
        float tx = 0.f, ty = 0.f, tz = 0.f;
#pragma unroll 16
        for (int jj = 0; jj < kJ; ++jj) {
            const float4 b = tile[part](jj);
            const float dx = b.x - px, dy = b.y - py, dz = b.z - pz;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
            const float rinv = rsqrtf(r2);
            const float s = b.w * (rinv * rinv * rinv);
            tx = fmaf(dx, s, tx);
            ty = fmaf(dy, s, ty);
            tz = fmaf(dz, s, tz);
        }
        ax += tx;
        ay += ty;
        az += tz;
        __syncthreads();
    }
    partial[part][li] = make_float3(ax, ay, az);
    __syncthreads();
    if (part == 0 && i < n) {
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
    nbody_update<KIND><<<blocks, kI * kParts, 0, stream>>>(v, eps * eps, dt, chunk);
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
