// layout.cuh -- arguments of the layout-building kernels (layout.cu, dem.cu).
#pragma once

#include "common.cuh"

namespace lbmdem {

struct PaintArgs {
    const double* X;
    const double* R;
    int nx, ny, nz, px;
    double skin;
    int32_t* owner;  // null: keep the current owner map (re-layout)
    unsigned long long* best;  // per node: smallest |y - X|^2 / R^2 (FP64 bits)
    uint8_t* deep;
    uint8_t* band;
};

struct LayoutArgs {
    int nx, ny, nz, nw;
    const int32_t* owner;
    const uint8_t* deep;
    const uint8_t* band;
    uint4* rec;
    uint32_t* maskB;
    uint32_t* cntA;
    uint32_t* cntB;
    uint32_t* coord;
};

struct SurfArgs {
    Lat L;
    const double* X;
    const double* R;
    double reach_extra;
    double skin;
    const int32_t* owner;   // map at layout time
    const uint8_t* band;    // band flags at layout time
    uint32_t* count;        // [n * LINK_GROUPS] links per (sphere, direction, maybe), padded
                            // to 32; the last group of a sphere also holds the padding to LINK_WARP
    const uint32_t* offset; // exclusive scan of count
    uint2* link;
    uint32_t* warp_p;
    uint8_t* chunk_dir;     // direction of every 32-record chunk (4 per warp)
    uint32_t* nlink;        // total link records before padding (accumulated)
};

struct CellGrid {
    int3 nc;        // cells per axis
    double3 lo, h;  // origin (x only) and cell size
    double3 L;      // box lengths (periodic axes)
    int px;
};

struct NbBuild {
    const double* X;
    const double* R;
    int n, nbmax;
    double skin;
    CellGrid G;
    const int* start;
    const int* order;
    int* cnt;
    int* nj;
    int8_t* nsh;     // [n*nbmax*4] image shift in box lengths
    float4* dref;    // xyz: X_ref_j + shift - X_ref_i; w: (R_i + R_j)^2 - |xyz|^2 (FP64-exact)
    float4* ft;
    const int* old_cnt;
    const int* old_j;
    const int8_t* old_sh;
    const float4* old_ft;
    uint32_t* status;
};

struct BandCand {
    const double* X;
    const double* R;
    double skin;
    CellGrid G;
    const int* start;
    const int* order;
    const uint32_t* coord;
    int4* cand;
    float* slack;
    uint32_t n;
    uint32_t* status;
    uint8_t* band_dense;   // per lattice node: 1 = one candidate sphere, 2 = several
    int nx, ny, nz;
};

void fill_i32(int32_t* p, int32_t v, size_t n, cudaStream_t s);
void exclusive_scan(const uint32_t* in, uint32_t* out, size_t n, uint32_t* tmp, cudaStream_t s);
size_t scan_tmp_size(size_t n);
void launch_paint(const PaintArgs& A, int n, size_t N, cudaStream_t s);
void launch_words(const LayoutArgs& A, cudaStream_t s);
void launch_words_bases(const LayoutArgs& A, uint32_t nA, cudaStream_t s);
void launch_coords(const LayoutArgs& A, uint32_t nA, uint32_t nSpad, uint32_t* fbits, cudaStream_t s);
void launch_gather_old(const Lat& Lnew, const Lat& Lold, cudaStream_t s);
void launch_band_collect(const LayoutArgs& A, uint32_t* band_coord, uint32_t* count, uint32_t cap,
                         cudaStream_t s);
void launch_surf_count(const SurfArgs& A, int n, cudaStream_t s);
void launch_surf_fill(const SurfArgs& A, int n, cudaStream_t s);

// dem.cu
void launch_cells(const double* X, int n, const CellGrid& G, int* cell_of, int* count, int* start,
                  int* fill, int* order, uint32_t* scan_tmp, cudaStream_t s);
void launch_nb_build(const NbBuild& B, cudaStream_t s);
void launch_band_cand(const BandCand& B, cudaStream_t s);
constexpr int SLACK_HIST = 1024 + 1;  // bucket counts (+ total) of launch_band_sort
void launch_band_sort(const uint32_t* coord, const int4* cand, const float* slack, uint32_t n, double skin,
                      uint32_t* hist, uint32_t* scan_tmp, uint32_t* coord2, int4* cand2, float* slack2,
                      cudaStream_t s);
void launch_rebase(double* Xref, float4* dX, float4* dXc, int n, cudaStream_t s);

}  // namespace lbmdem
