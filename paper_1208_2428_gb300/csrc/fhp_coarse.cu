// fhp_coarse.cu -- block coarse-graining of the bit-plane lattice.
//
// For each B x B block (B a multiple of 32, so a block row is B/32 whole
// words) one warp counts, over the fluid nodes of the block, how many carry
// each of the seven particles (population counts of plane & ~solid), the
// number of fluid nodes, and the mass; it then derives density and mean
// particle velocity in double precision:
//   rho = mass / fluid, ux = jx2 / (2 mass), uy = (sqrt(3)/2) jy / mass,
// with the integer momenta jx2 = sum_i n_i 2cos(theta_i) and
// jy = sum_i n_i sgn(sin(theta_i)), theta_i = (i-2)*60 degrees.
#include "fhp_internal.h"

namespace fhp {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kBlock = 256;

template <bool SOLID>
__global__ void __launch_bounds__(kBlock) coarse_kernel(Geometry g, const uint32_t* __restrict__ state,
                                                        const uint32_t* __restrict__ solid, int B,
                                                        int32_t* __restrict__ counts,
                                                        float* __restrict__ rho,
                                                        float* __restrict__ ux,
                                                        float* __restrict__ uy) {
    const int lane = threadIdx.x & 31;
    const int nbx = g.W / B, nby = g.H / B;
    const long long cell = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (cell >= (long long)nbx * nby) return;  // whole warp leaves together
    const int by = (int)(cell / nbx), bx = (int)(cell - (long long)by * nbx);
    const int wpr = B / 32;  // words per block row
    const int items = B * wpr;
    unsigned n[7] = {0, 0, 0, 0, 0, 0, 0};
    unsigned fluid = 0;
    for (int it = lane; it < items; it += 32) {
        const int yy = by * B + it / wpr;
        const int ww = bx * wpr + it % wpr;
        const size_t off = (size_t)yy * g.Pq + ww;
        const uint32_t f = SOLID ? ~solid[off] : 0xFFFFFFFFu;
        fluid += __popc(f);
#pragma unroll
        for (int k = 0; k < 7; ++k) n[k] += __popc(state[(size_t)k * g.plane_words + off] & f);
    }
#pragma unroll
    for (int k = 0; k < 7; ++k) n[k] = __reduce_add_sync(kFull, n[k]);
    fluid = __reduce_add_sync(kFull, fluid);
    if (lane != 0) return;
    long long mass = 0;
    for (int k = 0; k < 7; ++k) mass += n[k];
    const long long jx2 = -(long long)n[0] + n[1] + 2LL * n[2] + n[3] - (long long)n[4] - 2LL * n[5];
    const long long jy = -(long long)n[0] - (long long)n[1] + n[3] + n[4];
    int32_t* c = counts + (size_t)cell * 9;
    for (int k = 0; k < 7; ++k) c[k] = (int32_t)n[k];
    c[7] = (int32_t)fluid;
    c[8] = (int32_t)mass;
    const double half_sqrt3 = sqrt(3.0) * 0.5;
    const double r = fluid ? (double)mass / (double)fluid : 0.0;
    const double vx = mass ? (double)jx2 / (2.0 * (double)mass) : 0.0;
    const double vy = mass ? half_sqrt3 * (double)jy / (double)mass : 0.0;
    rho[cell] = __double2float_rn(r);
    ux[cell] = __double2float_rn(vx);
    uy[cell] = __double2float_rn(vy);
}

}  // namespace

cudaError_t launch_coarse_grain(const Geometry& g, const uint32_t* state, const uint32_t* solid,
                                bool has_solid, int B, int32_t* counts, float* rho, float* ux,
                                float* uy, cudaStream_t stream) {
    const long long cells = (long long)(g.W / B) * (g.H / B);
    const unsigned grid = (unsigned)((cells * 32 + kBlock - 1) / kBlock);
    if (has_solid)
        coarse_kernel<true><<<grid, kBlock, 0, stream>>>(g, state, solid, B, counts, rho, ux, uy);
    else
        coarse_kernel<false><<<grid, kBlock, 0, stream>>>(g, state, solid, B, counts, rho, ux, uy);
    return cudaGetLastError();
}

}  // namespace fhp
