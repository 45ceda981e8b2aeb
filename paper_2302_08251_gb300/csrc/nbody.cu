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

// Access instrumentation (Sec. 4).  CM = 1: one global atomic increment per
// access (the paper's scheme); CM = 2: per-block shared-memory counters,
// added to the global ones once per block (same counts, far fewer global
// atomics).  HEAT: one global atomic per granule an access touches.
template <int KIND, int CM, bool HEAT>
__device__ __forceinline__ void note(const ParticleView& v, const NbodyInstr& in, unsigned long long* block_counts,
                                     int f, uint32_t i, bool write)
{
    const int c = f + (write ? 7 : 0);
    if (CM == 1) atomicAdd(&in.counts[c], 1ull);
    if (CM == 2) atomicAdd(&block_counts[c], 1ull);
    if (HEAT) {
        const uint64_t off = in.boff[f] + Addr<KIND>::off(v, i);
        for (uint64_t k = off >> in.gshift; k <= (off + 3u) >> in.gshift; ++k)
            atomicAdd(&in.heat[in.hstart[f] + k], 1ull);
    }
}

template <int KIND, int CM, bool HEAT>
__device__ __forceinline__ float ld_i(const ParticleView& v, const NbodyInstr& in, unsigned long long* bc, int f,
                                      uint32_t i)
{
    if (CM != 0 || HEAT) note<KIND, CM, HEAT>(v, in, bc, f, i, false);
    return ld_leaf<KIND>(v, f, i);
}

template <int KIND, int CM, bool HEAT>
__device__ __forceinline__ void st_i(const ParticleView& v, const NbodyInstr& in, unsigned long long* bc, int f,
                                     uint32_t i, float x)
{
    if (CM != 0 || HEAT) note<KIND, CM, HEAT>(v, in, bc, f, i, true);
    st_leaf<KIND>(v, f, i, x);
}

template <int CM>
__device__ __forceinline__ void block_counts_init(unsigned long long* bc)
{
    if (CM == 2 && threadIdx.x < 14) bc[threadIdx.x] = 0ull;
}

// After a __syncthreads: add the block's counters to the global ones.
template <int CM>
__device__ __forceinline__ void block_counts_flush(const NbodyInstr& in, const unsigned long long* bc)
{
    if (CM == 2 && threadIdx.x < 14 && bc[threadIdx.x] != 0ull) atomicAdd(&in.counts[threadIdx.x], bc[threadIdx.x]);
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
template <int KIND, int CM = 0, bool HEAT = false>
__global__ void __launch_bounds__(kW * kParts) nbody_update(const ParticleView v, float eps2, float dt,
                                                            uint32_t chunk, const NbodyInstr in)
{
    __shared__ StaticBodyTile<kJ> tile[kParts];
    __shared__ float3 partial[kParts][kI];
    __shared__ unsigned long long bc[14];
    const uint32_t lane = threadIdx.x % kW;
    const uint32_t part = threadIdx.x / kW;
    const uint32_t i0 = blockIdx.x * kI + lane, i1 = i0 + kW;
    const uint32_t n = v.n;
    block_counts_init<CM>(bc);
    if (CM == 2) __syncthreads();

    // the block's own particles are read by slice 0 only (once each)
    float p0x = 0.f, p0y = 0.f, p0z = 0.f, p1x = 0.f, p1y = 0.f, p1z = 0.f;
    if (part == 0) {
        if (i0 < n) {
            p0x = ld_i<KIND, CM, HEAT>(v, in, bc, 0, i0);
            p0y = ld_i<KIND, CM, HEAT>(v, in, bc, 1, i0);
            p0z = ld_i<KIND, CM, HEAT>(v, in, bc, 2, i0);
        }
        if (i1 < n) {
            p1x = ld_i<KIND, CM, HEAT>(v, in, bc, 0, i1);
            p1y = ld_i<KIND, CM, HEAT>(v, in, bc, 1, i1);
            p1z = ld_i<KIND, CM, HEAT>(v, in, bc, 2, i1);
        }
        partial[0][lane] = make_float3(p0x, p0y, p0z);
        partial[0][lane + kW] = make_float3(p1x, p1y, p1z);
    }
    __syncthreads();
    if (part != 0) {
        const float3 q0 = partial[0][lane], q1 = partial[0][lane + kW];
        p0x = q0.x; p0y = q0.y; p0z = q0.z;
        p1x = q1.x; p1y = q1.y; p1z = q1.z;
    }
    __syncthreads();
    float a0x = 0.f, a0y = 0.f, a0z = 0.f, a1x = 0.f, a1y = 0.f, a1z = 0.f;
    const uint32_t j0 = part * chunk;
    for (uint32_t jt = 0; jt < chunk; jt += kJ) {
#pragma unroll
        for (int r = 0; r < kJ / kW; ++r) {
            const uint32_t jl = jt + lane + r * kW;
            const uint32_t j = j0 + jl;
            float4 q = make_float4(0.f, 0.f, 0.f, 0.f);  // zero mass beyond n
            if (j < n && jl < chunk)
                q = make_float4(ld_i<KIND, CM, HEAT>(v, in, bc, 0, j), ld_i<KIND, CM, HEAT>(v, in, bc, 1, j),
                                ld_i<KIND, CM, HEAT>(v, in, bc, 2, j), ld_i<KIND, CM, HEAT>(v, in, bc, 6, j));
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
            st_i<KIND, CM, HEAT>(v, in, bc, 3, i, fmaf(dt, sx, ld_i<KIND, CM, HEAT>(v, in, bc, 3, i)));
            st_i<KIND, CM, HEAT>(v, in, bc, 4, i, fmaf(dt, sy, ld_i<KIND, CM, HEAT>(v, in, bc, 4, i)));
            st_i<KIND, CM, HEAT>(v, in, bc, 5, i, fmaf(dt, sz, ld_i<KIND, CM, HEAT>(v, in, bc, 5, i)));
        }
    }
    if (CM == 2) {
        __syncthreads();
        block_counts_flush<CM>(in, bc);
    }
}

template <int KIND, int CM = 0, bool HEAT = false>
__global__ void nbody_move(const ParticleView v, float dt, const NbodyInstr in)
{
    __shared__ unsigned long long bc[14];
    block_counts_init<CM>(bc);
    if (CM == 2) __syncthreads();
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < v.n) {
        for (int k = 0; k < 3; ++k) {
            const float vel = ld_i<KIND, CM, HEAT>(v, in, bc, 3 + k, i);
            const float pos = ld_i<KIND, CM, HEAT>(v, in, bc, k, i);
            st_i<KIND, CM, HEAT>(v, in, bc, k, i, fmaf(dt, vel, pos));
        }
    }
    if (CM == 2) {
        __syncthreads();
        block_counts_flush<CM>(in, bc);
    }
}

template <int KIND, int CM = 0, bool HEAT = false>
static cudaError_t launch_kind(const ParticleView& v, float eps, float dt, cudaStream_t stream,
                               const NbodyInstr& in = NbodyInstr{})
{
    const uint32_t n = v.n;
    uint32_t chunk = (n + kParts - 1) / kParts;
    chunk = (chunk + kJ - 1) / kJ * kJ;
    const uint32_t blocks = (n + kI - 1) / kI;
    nbody_update<KIND, CM, HEAT><<<blocks, kW * kParts, 0, stream>>>(v, eps * eps, dt, chunk, in);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    nbody_move<KIND, CM, HEAT><<<(n + 255) / 256, 256, 0, stream>>>(v, dt, in);
    return cudaGetLastError();
}

// Instrumented steps use the runtime address function; the arithmetic, and
// so every result bit, is the plain step's.
cudaError_t launch_nbody_instrumented(const ParticleView& v, const NbodyInstr& in, float eps, float dt,
                                      cudaStream_t stream)
{
    if (v.n == 0) return cudaSuccess;
    const bool heat = in.heat != nullptr;
    const int cm = in.counts ? in.count_mode : 0;
    if (cm == 1) return heat ? launch_kind<PV_GENERIC, 1, true>(v, eps, dt, stream, in)
                             : launch_kind<PV_GENERIC, 1, false>(v, eps, dt, stream, in);
    if (cm == 2) return heat ? launch_kind<PV_GENERIC, 2, true>(v, eps, dt, stream, in)
                             : launch_kind<PV_GENERIC, 2, false>(v, eps, dt, stream, in);
    return heat ? launch_kind<PV_GENERIC, 0, true>(v, eps, dt, stream, in)
                : launch_kind<PV_GENERIC, 0, false>(v, eps, dt, stream, in);
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
