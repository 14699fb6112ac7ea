// Aggregation multigrid preconditioner: data structures shared by the setup
// (vip_mg.cu) and the V-cycle inside the Krylov launch (vip_krylov.cu).
#pragma once

#include <stdint.h>

namespace vip {

constexpr int MG_MAXLEV = 16;
// Cells of the largest geometry on the coarsest level (solved exactly by its dense
// inverse).  Open domains take a larger exact coarse solve (fewer iterations); a
// closed domain's pinned constant mode makes large coarse operators nearly singular,
// so contexts with a closed geometry keep it small.
constexpr int MG_COARSEST_OPEN = 2200;
constexpr int MG_COARSEST_CLOSED = 64;

struct MgGeom {                   // background lattice of one geometry
    double h, x0, y0;
    int32_t periodic_x, periodic_y;
    int32_t nx[MG_MAXLEV + 1], ny[MG_MAXLEV + 1];  // level 0 = lattice, l >= 1 = cells
    int32_t sx[MG_MAXLEV + 1];    // row stride of level l (nx padded to a multiple of 32)
};

// One geometry's cell lattice on one coarse level: cell (x, y), x < nx, y < ny, is
// number off + y * sx + x.  Cells x in [nx, sx) and the tail of the geometry's
// block (its length is a multiple of 32) are padding: no stencil, never read.
// px, py flag periodic directions.
struct MgLevGeom {
    int64_t off;
    int32_t nx, ny, sx, px, py, pad;
};

// Block of 32 x th cells of one geometry (th = the level's tile height), processed
// by one CTA.
struct MgTile {
    int32_t g, x0, y0, pad;
};

struct MgLevel {                  // coarse level (all geometries concatenated)
    int64_t n = 0;                // cells incl. padding (a multiple of 32)
    int32_t *cgeom = nullptr, *cx = nullptr, *cy = nullptr;  // cx = -1: padding
    int64_t* off = nullptr;       // [G] first cell of each geometry
    int32_t* nbr = nullptr;       // [25][n] neighbour cell of each 5x5 offset (-1: none)
    int32_t* parent = nullptr;    // [n] cell of the next level (-1: padding)
    int64_t* child = nullptr;     // [4][n] cells of the level above (-1: none)
    double* coef = nullptr;       // [25][n] Galerkin stencil (setup layout)
    double* coefs = nullptr;      // the same, sliced: [n/32][25][32] (V-cycle layout)
    float* coefs32 = nullptr;     // coefs rounded to FP32 (the FP32 V-cycle)
    double* dinv = nullptr;       // [n] l1-Jacobi scaling (0 for empty and padding cells)
    double* wdinv = nullptr;      // [n] omega * dinv (the smoother's step)
    float* wdinv32 = nullptr;     // [n] omega * dinv rounded to FP32
    uint8_t* ring = nullptr;      // [n/32] 1 if a cell of the slice has a nonzero outside its 3 x 3 core
    MgLevGeom* lg = nullptr;      // [G] lattice of each geometry on this level
    MgTile* tiles = nullptr;      // 32 x th tiles covering every geometry's lattice
    int64_t ntiles = 0;
    int th = 32;                  // tile height (32, 16, 8, 4 or 2 rows)
    void *x = nullptr, *b = nullptr, *y = nullptr;  // vectors (FP64 or FP32 view)
};

struct Multigrid {
    bool built = false;
    int nlev = 0;                 // coarse levels 1..nlev
    MgGeom* geom = nullptr;
    MgLevel lev[MG_MAXLEV + 1];
    int32_t* agg = nullptr;       // [R] level-1 cell of a fine row (-1: none)
    int64_t* cptr = nullptr;      // [n1+1] fine rows of each level-1 cell
    int32_t* crow = nullptr;
    double* fdinv = nullptr;      // [R] l1-Jacobi scaling of the fine operator
    double* fwdinv = nullptr;     // [R] omega * fdinv
    float* fwdinv32 = nullptr;    // [R] omega * fdinv rounded to FP32
    void* fr = nullptr;           // [R] fine residual scratch
    void* fx = nullptr;           // [R] fine smoothing scratch
    double* cinv = nullptr;       // dense inverse of each geometry's coarsest operator (row-major)
    float* cinv32 = nullptr;      // the same rounded to FP32
    int64_t* cinv_off = nullptr;  // [G] offset of geometry g's block in cinv
    int64_t cinv_entries = 0;     // entries of all geometries' coarsest inverses
    int ngeom = 0;
    float omega = 1.0f;           // smoother damping (vip_set_multigrid / vip_autotune)
    float corr = 1.5f;            // scaling of the coarse-grid correction
    float scaled_omega = -1.0f;   // the omega that fwdinv and wdinv hold
};

// Device view of the hierarchy with vectors, operators and arithmetic in precision
// T (FP64, or FP32 copies of every operator for the FP32 V-cycle).
template <class T>
struct MgDev {
    int nlev;
    int ngeom;
    const int32_t* agg;
    const int64_t* cptr;
    const int32_t* crow;
    const T* fwdinv;        // omega * fine l1-Jacobi scaling
    T* fr;
    T* fx;
    int64_t n[MG_MAXLEV + 1];
    int64_t ntiles[MG_MAXLEV + 1];
    const MgLevGeom* lg[MG_MAXLEV + 1];
    const MgTile* tiles[MG_MAXLEV + 1];
    const T* coefs[MG_MAXLEV + 1];            // sliced stencils
    const uint8_t* ring[MG_MAXLEV + 1];       // slices whose stencils reach beyond 3 x 3
    int32_t th[MG_MAXLEV + 1];                // tile heights
    const T* wdinv[MG_MAXLEV + 1];            // omega * l1-Jacobi scaling
    T* x[MG_MAXLEV + 1];
    T* b[MG_MAXLEV + 1];
    T* y[MG_MAXLEV + 1];
    float corr;        // scaling of the coarse-grid correction (piecewise-constant prolongation)
    const T* cinv;
    const int64_t* cinv_off;
};

}  // namespace vip
