// fhp_pack.cu -- conversion between node bytes (arXiv:1208.2428 Section 2,
// Fig. 1: bits 0-5 movers, bit 6 rest, bit 7 solid) and bit-planes, and the
// obstacle map.  One warp converts one 32-node word at a time: lane j holds
// node 32w + j and __ballot_sync gathers bit b of the 32 nodes into plane b.
#include <cmath>

#include "fhp_device.cuh"
#include "fhp_internal.h"

namespace fhp {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kBlock = 256;

unsigned grid_for(size_t warps) {
    size_t blocks = (warps * 32 + kBlock - 1) / kBlock;
    if (blocks > 65535u * 16u) blocks = 65535u * 16u;  // grid-stride loop covers the rest
    return (unsigned)(blocks ? blocks : 1);
}

__global__ void __launch_bounds__(kBlock) pack_kernel(Geometry g, const uint8_t* __restrict__ bytes,
                                                      uint32_t* __restrict__ state,
                                                      uint32_t* __restrict__ solid,
                                                      unsigned int* __restrict__ any_solid) {
    const int lane = threadIdx.x & 31;
    const size_t nwarps = ((size_t)gridDim.x * blockDim.x) >> 5;
    const size_t total = (size_t)g.H * g.Pq;
    for (size_t item = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; item < total;
         item += nwarps) {
        const int y = (int)(item / g.Pq);
        const int w = (int)(item - (size_t)y * g.Pq);
        uint32_t v = 0;
        if (w < g.Wq) v = bytes[(size_t)y * g.W + 32 * w + lane];
        uint32_t mine = 0;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const uint32_t plane_word = __ballot_sync(kFull, (v >> b) & 1u);
            if (lane == b) mine = plane_word;
        }
        const size_t off = (size_t)y * g.Pq + w;
        if (lane < 7) state[(size_t)lane * g.plane_words + off] = mine;
        if (lane == 7) {
            solid[off] = mine;
            if (mine) atomicOr(any_solid, 1u);
        }
    }
}

__global__ void __launch_bounds__(kBlock) unpack_kernel(Geometry g, const uint32_t* __restrict__ state,
                                                        const uint32_t* __restrict__ solid,
                                                        uint8_t* __restrict__ bytes) {
    const int lane = threadIdx.x & 31;
    const size_t nwarps = ((size_t)gridDim.x * blockDim.x) >> 5;
    const size_t total = (size_t)g.H * g.Wq;
    for (size_t item = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; item < total;
         item += nwarps) {
        const int y = (int)(item / g.Wq);
        const int w = (int)(item - (size_t)y * g.Wq);
        const size_t off = (size_t)y * g.Pq + w;
        uint32_t byte = ((solid[off] >> lane) & 1u) << 7;
#pragma unroll
        for (int b = 0; b < 7; ++b) byte |= ((state[(size_t)b * g.plane_words + off] >> lane) & 1u) << b;
        bytes[(size_t)y * g.W + 32 * w + lane] = (uint8_t)byte;
    }
}

__global__ void __launch_bounds__(kBlock) obstacle_kernel(Geometry g, const uint8_t* __restrict__ mask,
                                                          uint32_t* __restrict__ state,
                                                          uint32_t* __restrict__ solid,
                                                          unsigned int* __restrict__ any_solid) {
    const int lane = threadIdx.x & 31;
    const size_t nwarps = ((size_t)gridDim.x * blockDim.x) >> 5;
    const size_t total = (size_t)g.H * g.Pq;
    for (size_t item = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; item < total;
         item += nwarps) {
        const int y = (int)(item / g.Pq);
        const int w = (int)(item - (size_t)y * g.Pq);
        bool s = false;
        if (w < g.Wq) s = mask[(size_t)y * g.W + 32 * w + lane] != 0;
        const uint32_t word = __ballot_sync(kFull, s);
        const size_t off = (size_t)y * g.Pq + w;
        if (lane < 7 && word) state[(size_t)lane * g.plane_words + off] &= ~word;
        if (lane == 7) {
            solid[off] = word;
            if (word) atomicOr(any_solid, 1u);
        }
    }
}

// Generated initial state: for word w of row y and bit b, four Philox blocks
// (counter (w, y, b, j), j = 0..3, under the init key) give the 32 nodes'
// 16-bit uniforms -- node i takes block i / 8, output word (i mod 8) / 2,
// half i mod 2 -- and the node's bit b is set iff its uniform < P.  Solid
// nodes end without particles.
__global__ void __launch_bounds__(kBlock) init_kernel(Geometry g, uint32_t* __restrict__ state,
                                                      const uint32_t* __restrict__ solid, bool has_solid,
                                                      Key2 key, uint32_t P) {
    const size_t total = (size_t)g.H * g.Pq;
    for (size_t item = (size_t)blockIdx.x * blockDim.x + threadIdx.x; item < total;
         item += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(item / g.Pq);
        const int w = (int)(item - (size_t)y * g.Pq);
        const size_t off = (size_t)y * g.Pq + w;
        if (w >= g.Wq) {
            for (int b = 0; b < 7; ++b) state[(size_t)b * g.plane_words + off] = 0u;
            continue;
        }
        const uint32_t fluid = has_solid ? ~solid[off] : 0xFFFFFFFFu;
        for (int b = 0; b < 7; ++b) {
            uint32_t word = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint4 r = philox4x32_10(make_uint4((uint32_t)w, (uint32_t)y, (uint32_t)b, (uint32_t)j), key);
                const uint32_t outs[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const uint32_t u = (k & 1) ? (outs[k >> 1] >> 16) : (outs[k >> 1] & 0xFFFFu);
                    word |= (u < P ? 1u : 0u) << (8 * j + k);
                }
            }
            state[(size_t)b * g.plane_words + off] = word & fluid;
        }
    }
}

// Obstacles from shapes: one thread per word; a node is solid if any shape
// covers it (discs: squared distance in index coordinates, exact in 64-bit
// integers; row bands).
__global__ void __launch_bounds__(kBlock) shape_kernel(Geometry g, ShapeList shapes, uint32_t* __restrict__ state,
                                                       uint32_t* __restrict__ solid, unsigned int* any_solid) {
    const size_t total = (size_t)g.H * g.Pq;
    for (size_t item = (size_t)blockIdx.x * blockDim.x + threadIdx.x; item < total;
         item += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(item / g.Pq);
        const int w = (int)(item - (size_t)y * g.Pq);
        uint32_t word = 0;
        if (w < g.Wq) {
            for (int k = 0; k < shapes.n; ++k) {
                const Shape sh = shapes.s[k];
                if (sh.kind == 2) {
                    if (y >= sh.a && y < sh.b) word = 0xFFFFFFFFu;
                } else if (sh.kind == 1) {
                    const long long dy = (long long)y - sh.b;
                    const long long r2 = (long long)sh.c * sh.c - dy * dy;
                    if (r2 < 0) continue;
                    for (int i = 0; i < 32; ++i) {
                        const long long dx = (long long)(32 * w + i) - sh.a;
                        if (dx * dx <= r2) word |= 1u << i;
                    }
                }
            }
        }
        const size_t off = (size_t)y * g.Pq + w;
        solid[off] = word;
        if (word) {
            for (int b = 0; b < 7; ++b) state[(size_t)b * g.plane_words + off] &= ~word;
            if (any_solid) atomicOr(any_solid, 1u);
        }
    }
}

}  // namespace

cudaError_t launch_obstacle_shapes(const Geometry& g, const ShapeList& shapes, uint32_t* state, uint32_t* solid,
                                   unsigned int* device_any_solid, cudaStream_t stream) {
    shape_kernel<<<grid_for((size_t)g.H * g.Pq / 32 + 1), kBlock, 0, stream>>>(g, shapes, state, solid,
                                                                               device_any_solid);
    return cudaGetLastError();
}

cudaError_t launch_init_random(const Geometry& g, uint32_t* state, const uint32_t* solid, bool has_solid,
                               uint64_t seed, double density, cudaStream_t stream) {
    const double scaled = density * 65536.0;
    uint32_t P;
    if (!(scaled > 0.0)) P = 0;
    else if (scaled >= 65536.0) P = 65536;
    else P = (uint32_t)std::nearbyint(scaled);  // nearest, ties to even
    const Key2 key{(uint32_t)seed ^ 0x9E3779B9u, (uint32_t)(seed >> 32) ^ 0x7F4A7C15u};
    init_kernel<<<grid_for((size_t)g.H * g.Pq / 32 + 1), kBlock, 0, stream>>>(g, state, solid, has_solid, key, P);
    return cudaGetLastError();
}

cudaError_t launch_pack(const Geometry& g, const uint8_t* bytes, uint32_t* state, uint32_t* solid,
                        unsigned int* device_any_solid, cudaStream_t stream) {
    pack_kernel<<<grid_for((size_t)g.H * g.Pq), kBlock, 0, stream>>>(g, bytes, state, solid,
                                                                    device_any_solid);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const Geometry& g, const uint32_t* state, const uint32_t* solid,
                          uint8_t* bytes, cudaStream_t stream) {
    unpack_kernel<<<grid_for((size_t)g.H * g.Wq), kBlock, 0, stream>>>(g, state, solid, bytes);
    return cudaGetLastError();
}

cudaError_t launch_load_obstacles(const Geometry& g, const uint8_t* mask, uint32_t* state,
                                  uint32_t* solid, unsigned int* device_any_solid,
                                  cudaStream_t stream) {
    obstacle_kernel<<<grid_for((size_t)g.H * g.Pq), kBlock, 0, stream>>>(g, mask, state, solid,
                                                                        device_any_solid);
    return cudaGetLastError();
}

}  // namespace fhp
