// Aggregation multigrid preconditioner: data structures shared by the setup
// (vip_mg.cu) and the V-cycle inside the Krylov launch (vip_krylov.cu).
#pragma once

#include <stdint.h>

namespace vip {

constexpr int MG_MAXLEV = 16;
constexpr int MG_COARSEST = 64;   // cells of the largest geometry on the coarsest level

struct MgGeom {                   // background lattice of one geometry
    double h, x0, y0;
    int32_t periodic_x, periodic_y;
    int32_t nx[MG_MAXLEV + 1], ny[MG_MAXLEV + 1];  // level 0 = lattice, l >= 1 = cells
};

struct MgLevel {                  // coarse level (all geometries concatenated)
    int64_t n = 0;
    int32_t *cgeom = nullptr, *cx = nullptr, *cy = nullptr;
    int64_t* off = nullptr;       // [G] first cell of each geometry
    int32_t* nbr = nullptr;       // [25][n] neighbour cell of each 5x5 offset (-1: none)
    int32_t* parent = nullptr;    // [n] cell of the next level
    int64_t* child = nullptr;     // [4][n] cells of the level above (-1: none)
    double* coef = nullptr;       // [25][n] Galerkin stencil
    float* coef32 = nullptr;
    double* dinv = nullptr;       // [n] inverse diagonal (0 for empty cells)
    float* dinv32 = nullptr;
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
    double* fdinv = nullptr;      // [R] inverse diagonal of the fine operator
    float* fdinv32 = nullptr;
    void* fr = nullptr;           // [R] fine residual scratch
    void* fx = nullptr;           // [R] fine smoothing scratch
    double* cinv = nullptr;       // dense inverse of each geometry's coarsest operator
    int64_t* cinv_off = nullptr;  // [G] offset of geometry g's block in cinv
    int ngeom = 0;
};

// Device view of the hierarchy in precision T.
template <class T>
struct MgDev {
    int nlev;
    const int32_t* agg;
    const int64_t* cptr;
    const int32_t* crow;
    const T* fdinv;
    T* fr;
    T* fx;
    int64_t n[MG_MAXLEV + 1];
    const int32_t* nbr[MG_MAXLEV + 1];
    const int32_t* parent[MG_MAXLEV + 1];
    const int64_t* child[MG_MAXLEV + 1];
    const T* coef[MG_MAXLEV + 1];
    const T* dinv[MG_MAXLEV + 1];
    T* x[MG_MAXLEV + 1];
    T* b[MG_MAXLEV + 1];
    T* y[MG_MAXLEV + 1];
    float omega;       // Jacobi damping
    float corr;        // scaling of the coarse-grid correction (piecewise-constant prolongation)
    const double* cinv;
    const int64_t* cinv_off;
    const int64_t* coff;  // [G] first cell of each geometry on the coarsest level
    int ngeom;
};

}  // namespace vip
