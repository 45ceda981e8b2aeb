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
// Two traversals of the records (the paper leaves mapping-aware loops open
// in Sec. 5): the index traversal maps each record index through the mapping
// on every access; the blocks traversal follows the layout -- in the move, an
// AoSoA block's pos leaves are one run of 3 L floats updated from the vel run
// after it, and SoA leaves are walked four records per thread, in 16-byte
// accesses; in the update, addresses advance as (block, lane) cursors.
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
        if (KIND == PV_DIV) {
            const uint32_t b = i / v.lanes;
            return (uint64_t)b * v.bstride + (uint64_t)(i - b * v.lanes) * 4u;
        }
        return (uint64_t)(i >> v.lshift) * v.bstride + (uint64_t)(i & v.lmask) * 4u;
    }
};

// The blocks traversal's address: a (block, lane) cursor.  Placing it costs
// one division; moving it 32 records on costs an add and a compare.
struct Cursor {
    uint64_t off;
    uint32_t lane;
    __device__ __forceinline__ void at(const ParticleView& v, uint32_t i)
    {
        const uint32_t b = i / v.lanes;
        lane = i - b * v.lanes;
        off = (uint64_t)b * v.bstride + (uint64_t)lane * 4u;
    }
    __device__ __forceinline__ void next32(const ParticleView& v)
    {
        lane += v.step_lanes;
        off += v.step_off;
        if (lane >= v.lanes) {
            lane -= v.lanes;
            off += v.wrap_off;
        }
    }
};

__device__ __forceinline__ float ld_at(const ParticleView& v, int f, uint64_t off)
{
    return *reinterpret_cast<const float*>(v.base[f] + off);
}

__device__ __forceinline__ void st_at(const ParticleView& v, int f, uint64_t off, float x)
{
    *reinterpret_cast<float*>(v.base[f] + off) = x;
}

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

// 1 / sqrt(x) by the SFU's approximation.  x = |d|^2 + eps^2 >= eps^2 is never
// subnormal for a softening eps above 1e-19, so the flush-to-zero form is
// taken: it gives rsqrtf's result bits for every normal x and skips
// rsqrtf's subnormal-input handling (about 3.5 of 17 instructions per
// interaction).
__device__ __forceinline__ float rsqrt_normal(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Interaction of particle p with record b = {x, y, z, m}, summed into t.
__device__ __forceinline__ void interact(const float4 b, float px, float py, float pz, float eps2, float& tx,
                                         float& ty, float& tz)
{
    const float dx = b.x - px, dy = b.y - py, dz = b.z - pz;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
    const float rinv = rsqrt_normal(r2);
    const float s = b.w * (rinv * rinv * rinv);
    tx = fmaf(dx, s, tx);
    ty = fmaf(dy, s, ty);
    tz = fmaf(dz, s, tz);
}

// One warp per j slice: it stages kJ-record tiles of its slice with warp-
// level synchronisation only, and every lane interacts two particles (i and
// i + 32) with each staged record.
// TRAV = TRAVERSE_INDEX maps every access's record index through the
// mapping; TRAVERSE_BLOCKS walks (block, lane) cursors (uninstrumented only).
template <int KIND, int CM = 0, bool HEAT = false, int TRAV = TRAVERSE_INDEX>
__global__ void __launch_bounds__(kW * kParts) nbody_update(const ParticleView v, float eps2, float dt,
                                                            uint32_t chunk, const NbodyInstr in)
{
    static_assert(TRAV == TRAVERSE_INDEX || (CM == 0 && !HEAT), "instrumented steps use the index traversal");
    __shared__ StaticBodyTile<kJ> tile[kParts];
    __shared__ float3 partial[kParts][kI];
    __shared__ unsigned long long bc[14];
    const uint32_t lane = threadIdx.x % kW;
    const uint32_t part = threadIdx.x / kW;
    const uint32_t i0 = blockIdx.x * kI + lane, i1 = i0 + kW;
    const uint32_t n = v.n;
    block_counts_init<CM>(bc);
    if (CM == 2) __syncthreads();
    // record i (cursor c in the blocks traversal), leaf f
    auto ld = [&](int f, uint32_t i, const Cursor& c) -> float {
        if constexpr (TRAV == TRAVERSE_BLOCKS) return ld_at(v, f, c.off);
        else return ld_i<KIND, CM, HEAT>(v, in, bc, f, i);
    };
    auto st = [&](int f, uint32_t i, const Cursor& c, float x) {
        if constexpr (TRAV == TRAVERSE_BLOCKS) st_at(v, f, c.off, x);
        else st_i<KIND, CM, HEAT>(v, in, bc, f, i, x);
    };
    // cursors of the block's own records (placed again after the j loop, so
    // that they hold no registers through it)
    Cursor own[kIPT] = {};
    auto place_own = [&]() {
        if constexpr (TRAV == TRAVERSE_BLOCKS) {
            own[0].at(v, i0);
            own[1] = own[0];
            own[1].next32(v);
        }
    };
    if (part == 0) place_own();

    // the block's own particles are read by slice 0 only (once each)
    float p0x = 0.f, p0y = 0.f, p0z = 0.f, p1x = 0.f, p1y = 0.f, p1z = 0.f;
    if (part == 0) {
        if (i0 < n) {
            p0x = ld(0, i0, own[0]);
            p0y = ld(1, i0, own[0]);
            p0z = ld(2, i0, own[0]);
        }
        if (i1 < n) {
            p1x = ld(0, i1, own[1]);
            p1y = ld(1, i1, own[1]);
            p1z = ld(2, i1, own[1]);
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
    Cursor cj = {};
    if constexpr (TRAV == TRAVERSE_BLOCKS) cj.at(v, j0 + lane);
    for (uint32_t jt = 0; jt < chunk; jt += kJ) {
#pragma unroll
        for (int r = 0; r < kJ / kW; ++r) {
            const uint32_t jl = jt + lane + r * kW;
            const uint32_t j = j0 + jl;
            float4 q = make_float4(0.f, 0.f, 0.f, 0.f);  // zero mass beyond n
            if (j < n && jl < chunk) q = make_float4(ld(0, j, cj), ld(1, j, cj), ld(2, j, cj), ld(6, j, cj));
            tile[part](lane + r * kW) = q;
            if constexpr (TRAV == TRAVERSE_BLOCKS) cj.next32(v);
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
        place_own();
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
            st(3, i, own[h], fmaf(dt, sx, ld(3, i, own[h])));
            st(4, i, own[h], fmaf(dt, sy, ld(4, i, own[h])));
            st(5, i, own[h], fmaf(dt, sz, ld(5, i, own[h])));
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

// The blocks traversal of the move on SoA: four consecutive records of every
// leaf per thread, as 16-byte accesses when VEC (all six leaf arrays 16-byte
// aligned).
template <bool VEC>
__global__ void __launch_bounds__(256) nbody_move_soa(const ParticleView v, float dt)
{
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t i = 4u * q;
    if (i >= v.n) return;
    if (VEC && i + 4u <= v.n) {
        float4 p[3], w[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            p[k] = reinterpret_cast<const float4*>(v.base[k])[q];
            w[k] = reinterpret_cast<const float4*>(v.base[3 + k])[q];
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            p[k].x = fmaf(dt, w[k].x, p[k].x);
            p[k].y = fmaf(dt, w[k].y, p[k].y);
            p[k].z = fmaf(dt, w[k].z, p[k].z);
            p[k].w = fmaf(dt, w[k].w, p[k].w);
            reinterpret_cast<float4*>(v.base[k])[q] = p[k];
        }
        return;
    }
    const uint32_t e = min(i + 4u, v.n);
    for (uint32_t r = i; r < e; ++r)
        for (int k = 0; k < 3; ++k) {
            float* pk = reinterpret_cast<float*>(v.base[k]) + r;
            *pk = fmaf(dt, reinterpret_cast<const float*>(v.base[3 + k])[r], *pk);
        }
}

// The blocks traversal of the move on AoSoA with L lanes: thread row y of a
// CTA owns AoSoA block b; the block's pos leaves are one run of 3 L floats
// and its vel leaves the next 3 L, element for element, so the row updates
// the run in units (16-byte quads when VEC, i.e. L % 4 == 0; floats
// otherwise).  The last block holds n - full * L < L records; only its used
// lanes are touched.
template <bool VEC>
__global__ void __launch_bounds__(256) nbody_move_aosoa(const ParticleView v, float dt, uint32_t full)
{
    const uint32_t L = v.lanes;
    const uint32_t b = blockIdx.x * blockDim.y + threadIdx.y;
    uint8_t* const P = v.base[0] + (uint64_t)b * v.bstride;
    const uint32_t vel = 12u * L;  // bytes from the pos run to the vel run
    if (b < full) {
        if (VEC) {
            for (uint32_t u = threadIdx.x; u < 3u * L / 4u; u += blockDim.x) {
                float4 p = *reinterpret_cast<const float4*>(P + 16u * u);
                const float4 w = *reinterpret_cast<const float4*>(P + vel + 16u * u);
                p.x = fmaf(dt, w.x, p.x);
                p.y = fmaf(dt, w.y, p.y);
                p.z = fmaf(dt, w.z, p.z);
                p.w = fmaf(dt, w.w, p.w);
                *reinterpret_cast<float4*>(P + 16u * u) = p;
            }
        } else {
            for (uint32_t u = threadIdx.x; u < 3u * L; u += blockDim.x) {
                float* p = reinterpret_cast<float*>(P + 4u * u);
                *p = fmaf(dt, *reinterpret_cast<const float*>(P + vel + 4u * u), *p);
            }
        }
    } else if (b == full) {
        const uint32_t used = v.n - full * L;
        for (uint32_t u = threadIdx.x; u < 3u * L; u += blockDim.x) {
            if (u % L >= used) continue;
            float* p = reinterpret_cast<float*>(P + 4u * u);
            *p = fmaf(dt, *reinterpret_cast<const float*>(P + vel + 4u * u), *p);
        }
    }
}

template <int KIND, int CM = 0, bool HEAT = false, int TRAV = TRAVERSE_INDEX>
static cudaError_t launch_update(const ParticleView& v, float eps, float dt, cudaStream_t stream,
                                 const NbodyInstr& in = NbodyInstr{})
{
    const uint32_t n = v.n;
    uint32_t chunk = (n + kParts - 1) / kParts;
    chunk = (chunk + kJ - 1) / kJ * kJ;
    const uint32_t blocks = (n + kI - 1) / kI;
    nbody_update<KIND, CM, HEAT, TRAV><<<blocks, kW * kParts, 0, stream>>>(v, eps * eps, dt, chunk, in);
    return cudaGetLastError();
}

template <int KIND, int CM = 0, bool HEAT = false>
static cudaError_t launch_move(const ParticleView& v, float dt, cudaStream_t stream,
                               const NbodyInstr& in = NbodyInstr{})
{
    nbody_move<KIND, CM, HEAT><<<(v.n + 255) / 256, 256, 0, stream>>>(v, dt, in);
    return cudaGetLastError();
}

template <int KIND, int CM = 0, bool HEAT = false>
static cudaError_t launch_kind(const ParticleView& v, float eps, float dt, cudaStream_t stream,
                               const NbodyInstr& in = NbodyInstr{})
{
    const cudaError_t e = launch_update<KIND, CM, HEAT>(v, eps, dt, stream, in);
    if (e != cudaSuccess) return e;
    return launch_move<KIND, CM, HEAT>(v, dt, stream, in);
}

// Instrumented steps use the runtime address function; the arithmetic, and
// so every result bit, is the plain step's.
template <int KIND>
static cudaError_t launch_instrumented(const ParticleView& v, const NbodyInstr& in, float eps, float dt,
                                       cudaStream_t stream)
{
    const bool heat = in.heat != nullptr;
    const int cm = in.counts ? in.count_mode : 0;
    if (cm == 1) return heat ? launch_kind<KIND, 1, true>(v, eps, dt, stream, in)
                             : launch_kind<KIND, 1, false>(v, eps, dt, stream, in);
    if (cm == 2) return heat ? launch_kind<KIND, 2, true>(v, eps, dt, stream, in)
                             : launch_kind<KIND, 2, false>(v, eps, dt, stream, in);
    return heat ? launch_kind<KIND, 0, true>(v, eps, dt, stream, in)
                : launch_kind<KIND, 0, false>(v, eps, dt, stream, in);
}

cudaError_t launch_nbody_instrumented(const ParticleView& v, bool div, const NbodyInstr& in, float eps, float dt,
                                      cudaStream_t stream)
{
    if (v.n == 0) return cudaSuccess;
    return div ? launch_instrumented<PV_DIV>(v, in, eps, dt, stream)
               : launch_instrumented<PV_GENERIC>(v, in, eps, dt, stream);
}

// The plain step: the update with the index traversal (within a few per cent
// of the blocks traversal there, and fewer registers), the move with the
// blocks traversal (the faster one for this memory-bound phase).
cudaError_t launch_nbody(const ParticleView& v, int kind, int layout, float eps, float dt, cudaStream_t stream)
{
    if (v.n == 0) return cudaSuccess;
    const cudaError_t e = launch_nbody_update(v, kind, TRAVERSE_INDEX, eps, dt, stream);
    if (e != cudaSuccess) return e;
    return launch_nbody_move(v, kind, layout, TRAVERSE_BLOCKS, dt, stream);
}

cudaError_t launch_nbody_update(const ParticleView& v, int kind, int traversal, float eps, float dt,
                                cudaStream_t stream)
{
    if (v.n == 0) return cudaSuccess;
    if (traversal == TRAVERSE_BLOCKS) return launch_update<PV_GENERIC, 0, false, TRAVERSE_BLOCKS>(v, eps, dt, stream);
    switch (kind) {
    case PV_AOS: return launch_update<PV_AOS>(v, eps, dt, stream);
    case PV_SOA: return launch_update<PV_SOA>(v, eps, dt, stream);
    case PV_AOSOA32: return launch_update<PV_AOSOA32>(v, eps, dt, stream);
    case PV_DIV: return launch_update<PV_DIV>(v, eps, dt, stream);
    default: return launch_update<PV_GENERIC>(v, eps, dt, stream);
    }
}

cudaError_t launch_nbody_move(const ParticleView& v, int kind, int layout, int traversal, float dt,
                              cudaStream_t stream)
{
    if (v.n == 0) return cudaSuccess;
    if (traversal == TRAVERSE_BLOCKS && layout == 1) {
        bool vec = true;
        for (int f = 0; f < 6; ++f) vec = vec && (reinterpret_cast<uintptr_t>(v.base[f]) & 15u) == 0;
        const uint32_t grid = (v.n + 1023u) / 1024u;  // 256 threads x 4 records
        if (vec) nbody_move_soa<true><<<grid, 256, 0, stream>>>(v, dt);
        else nbody_move_soa<false><<<grid, 256, 0, stream>>>(v, dt);
        return cudaGetLastError();
    }
    if (traversal == TRAVERSE_BLOCKS && layout == 2) {
        const uint32_t L = v.lanes;
        const bool vec = L % 4u == 0 && (reinterpret_cast<uintptr_t>(v.base[0]) & 15u) == 0;
        const uint32_t units = vec ? 3u * L / 4u : 3u * L;
        const uint32_t bx = units < 256u ? units : 256u;
        const uint32_t by = 256u / bx;
        const uint32_t full = v.n / L;
        const uint32_t blocks = full + (v.n % L ? 1u : 0u);
        const dim3 block(bx, by);
        const uint32_t grid = (blocks + by - 1) / by;
        if (vec) nbody_move_aosoa<true><<<grid, block, 0, stream>>>(v, dt, full);
        else nbody_move_aosoa<false><<<grid, block, 0, stream>>>(v, dt, full);
        return cudaGetLastError();
    }
    // the index traversal; an AoS record is its own block, so AoS walks the same way in both
    switch (kind) {
    case PV_AOS: return launch_move<PV_AOS>(v, dt, stream);
    case PV_SOA: return launch_move<PV_SOA>(v, dt, stream);
    case PV_AOSOA32: return launch_move<PV_AOSOA32>(v, dt, stream);
    case PV_DIV: return launch_move<PV_DIV>(v, dt, stream);
    default: return launch_move<PV_GENERIC>(v, dt, stream);
    }
}

// FP32 fused multiply-add throughput probe: the roofline of the n-body
// update, which is bound by its FP32 arithmetic.  Every thread runs 16
// independent FMA chains for `iters` rounds (16 iters FMAs per thread); the
// chains' sum is stored only when it is exactly -1, which the inputs never
// give but the compiler cannot rule out, so no FMA is removed.
__global__ void __launch_bounds__(256) fma_probe_kernel(uint32_t iters, float* sink)
{
    float a[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = (float)(threadIdx.x + k) * 1e-6f;
    const float b = 0.9999999f, c = 1e-7f;
    for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 16; ++k) s += a[k];
    if (s == -1.0f) *sink = s;
}

cudaError_t launch_fma_probe(uint32_t iters, float* sink, uint64_t* fmas, cudaStream_t stream)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const uint32_t grid = (uint32_t)sms * 8u;  // 8 x 256 threads: every warp slot of an SM
    fma_probe_kernel<<<grid, 256, 0, stream>>>(iters, sink);
    *fmas = (uint64_t)grid * 256u * 16u * iters;
    return cudaGetLastError();
}

}  // namespace llgb
