// Device-side building blocks of the culled rollout (the voxel grid of the
// filter as a neighbour grid of S_W), shared by rollout_agents_culled
// (culled.cu) and the culled served loop (serve.cu).
//
// Neighbour index: S_W comes out of filter_cloud sorted by its linear key
// (i_z dims_y + i_y) dims_x + i_x, so the obstacles of a grid row (fixed
// i_y, i_z) with i_x in [a, b] lie in one index range.  wr[w] = the number
// of obstacles whose key is below 32 w (gmapp_grid_index); a row's range is
// [wr[klo / 32], wr[khi / 32 + 1]) with klo, khi the keys of its end cells --
// at most 31 cells of slack at each end, which the gate rejects.
#pragma once

#include "rollout_kernel.cuh"

namespace gmapp {

struct NeighbourGrid {
    const uint32_t *wr;  // [ceil(cells / 32) + 1]
    float lo[3], voxel;
    int32_t nx, ny, nz;
};

// Index range [i0, i1] of the cells whose extent meets [c - r, c + r] along
// one axis (clamped to the grid); empty when i0 > i1.
__device__ __forceinline__ void cell_span(float c, float r, float lo, float voxel, int n, int &i0,
                                          int &i1) {
    const float a = floorf((c - r - lo) / voxel), b = floorf((c + r - lo) / voxel);
    i0 = a < 0.0f ? 0 : (a >= static_cast<float>(n) ? n : static_cast<int>(a));
    i1 = b < 0.0f ? -1 : (b >= static_cast<float>(n) ? n - 1 : static_cast<int>(b));
}

// This thread's part of the Alg. 1 sum W and of min |d|^2 for an agent at p:
// the grid rows of the box of half-width `reach` around p are dealt to the
// NT threads of the CTA (rows whose (y, z) cells lie farther than the reach
// are skipped); every obstacle of a row's index range is evaluated with the
// gate d^2 <= G2 and the clamp max(|d| - R, eps).
template <int NT, bool CLEAR>
__device__ __forceinline__ void culled_terms(const float (&p)[3], float reach, float G2, float R,
                                             float eps, const NeighbourGrid &g, const float *ox,
                                             const float *oy, const float *oz, int tid, float &W,
                                             float &md2) {
    W = 0.0f;
    md2 = INFINITY;
    if (!(reach > 0.0f)) return;
    int x0, x1, y0, y1, z0, z1;
    cell_span(p[0], reach, g.lo[0], g.voxel, g.nx, x0, x1);
    cell_span(p[1], reach, g.lo[1], g.voxel, g.ny, y0, y1);
    cell_span(p[2], reach, g.lo[2], g.voxel, g.nz, z0, z1);
    const int ny_r = y1 - y0 + 1, nz_r = z1 - z0 + 1;
    const int rows = (x0 <= x1 && ny_r > 0 && nz_r > 0) ? ny_r * nz_r : 0;
    const float r2 = reach * reach;
    for (int r = tid; r < rows; r += NT) {
        const int iy = y0 + r % ny_r, iz = z0 + r / ny_r;
        // distance from p to the row's cells in (y, z)
        const float cy = g.lo[1] + static_cast<float>(iy) * g.voxel;
        const float cz = g.lo[2] + static_cast<float>(iz) * g.voxel;
        const float dy = fmaxf(fmaxf(cy - p[1], p[1] - (cy + g.voxel)), 0.0f);
        const float dz = fmaxf(fmaxf(cz - p[2], p[2] - (cz + g.voxel)), 0.0f);
        if (dy * dy + dz * dz > r2) continue;
        const uint32_t row =
            static_cast<uint32_t>(iz) * static_cast<uint32_t>(g.ny) + static_cast<uint32_t>(iy);
        const uint32_t klo = row * static_cast<uint32_t>(g.nx) + static_cast<uint32_t>(x0);
        const uint32_t khi = row * static_cast<uint32_t>(g.nx) + static_cast<uint32_t>(x1);
        const uint32_t j0 = __ldg(g.wr + (klo >> 5)), j1 = __ldg(g.wr + (khi >> 5) + 1);
        for (uint32_t j = j0; j < j1; ++j) {
            const float dx = p[0] - __ldg(ox + j), ey = p[1] - __ldg(oy + j),
                        ez = p[2] - __ldg(oz + j);
            const float d2 = fmaf(ez, ez, fmaf(ey, ey, dx * dx));
            const float s = fmaxf(fmaf(d2, rsqrt_approx(d2), -R), eps);
            if (d2 <= G2) W += rcp_approx(s);
            if (CLEAR) md2 = fminf(md2, d2);
        }
    }
}

// Fixed-order CTA reduction of (W, min |d|^2): warp butterflies, then the
// warps in order by thread 0 (the only thread whose result is defined).
template <int NT, bool CLEAR>
__device__ __forceinline__ void culled_reduce(float &W, float &md2, float *s_w, float *s_m) {
    constexpr int NW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    W = warp_sum(W);
    if (CLEAR) md2 = warp_min(md2);
    if (lane == 0) {
        s_w[warp] = W;
        s_m[warp] = md2;
    }
    __syncthreads();
    if (tid == 0) {
        float Wt = 0.0f, mt = INFINITY;
#pragma unroll
        for (int q = 0; q < NW; ++q) {
            Wt += s_w[q];
            mt = fminf(mt, s_m[q]);
        }
        W = Wt;
        md2 = mt;
    }
}

// Reach of an agent's gate in centre distance: s <= r_d  <=>  d <= r_d + R;
// rows are taken within it plus a margin far above FP32 rounding (negative:
// no gate can be met).
__device__ __forceinline__ float culled_reach(float rd, float R, float eps, float voxel) {
    return rd >= eps ? (rd + R) + 1e-3f * voxel : -1.0f;
}

}  // namespace gmapp
