// grid.cuh -- the float32 cell-key contract of the LR grid (declared in
// gs.h): cell side h, origin o and 1/h are float32 values fixed at create;
// the coordinate is floor((x - o) * (1/h)) in round-to-nearest without a
// fused multiply-add, clamped to the grid; the linear cell id is
// (cz * dy + cy) * dx + cx, offset by the scene's first cell.
#pragma once

#include <cuda_runtime.h>

#include "gs_internal.cuh"

// Twice the cell coordinate (the octant bit is the low bit), clamped.
__device__ __forceinline__ int grid_sub_coord(float x, float o, float inv_h, int dim)
{
    float a = __fmul_rn(__fsub_rn(x, o), inv_h);
    float f = floorf(__fmul_rn(a, 2.0f));
    if (!(f >= 0.0f)) return 0;
    if (f >= (float)(2 * dim - 1)) return 2 * dim - 1;
    return (int)f;
}

// Global cell id of a position in a scene.
__device__ __forceinline__ uint32_t grid_cell_of(const SceneDev& sc, float x, float y, float z)
{
    const GridDev& g = sc.g;
    const int sx = grid_sub_coord(x, g.ox, g.inv_h, g.dx);
    const int sy = grid_sub_coord(y, g.oy, g.inv_h, g.dy);
    const int sz = grid_sub_coord(z, g.oz, g.inv_h, g.dz);
    return sc.cell_off +
           ((uint32_t)(sz >> 1) * (uint32_t)g.dy + (uint32_t)(sy >> 1)) * (uint32_t)g.dx + (uint32_t)(sx >> 1);
}
