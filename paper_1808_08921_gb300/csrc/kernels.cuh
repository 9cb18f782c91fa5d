// kernels.cuh -- launch interfaces between the host orchestration (api.cu)
// and the kernel translation units.
#pragma once

#include "common.cuh"

namespace lbmdem {

// Fused monitors of the collide kernels.
struct Mon {
    double* acc;                    // [5] sum drho, sum j, fluid count (FP64)
    uint32_t* umax_bits;            // max |u|^2 as float bits
    uint32_t* status;
    double* probe_sum;              // [2 * capacity] (sum drho, count) per step, or null
    const unsigned long long* t_dev;
    uint32_t pA0, pA1, pB0, pB1;    // compact index ranges of the probe plane
};

struct Source {
    int waveform;
    double amp, omega, t0;
    long long t_n;
};

struct BC {
    int inlet, outlet;
    Source src;
    const unsigned long long* t_dev;
};

// Eq. 25 and Table 2 at time t (steps completed), in FP64 (evaluated once
// per block).
__device__ __forceinline__ double source_drho(const Source& S, unsigned long long t) {
    if (S.t_n >= 0 && (long long)t > S.t_n) return 0.0;
    double ph = S.omega * (double)t;
    switch (S.waveform) {
        case 0: return S.amp * sin(ph);
        case 1: return S.amp * (1.0 - cos(ph));
        case 2: return S.amp;
        case 3: {
            double a = 0.5 * S.omega * ((double)t - S.t0);  // pi f (t - t0), f = omega / 2 pi
            return S.amp * (1.0 - 2.0 * a * a) * exp(-a * a);
        }
    }
    return 0.0;
}

// Section 2.4, x-normal D3Q19 pressure face on deviations.  side 0: inlet
// (unknown c_x = +1), side 1: outlet (unknown c_x = -1).  Indices are the
// paper's d (1-based) minus one.
__device__ __forceinline__ void pressure_face(float g[Q], float drho_b, int side) {
    float rest = g[18] + g[2] + g[3] + g[4] + g[5] + g[14] + g[15] + g[16] + g[17];
    float Ny = 0.5f * (g[2] + g[14] + g[15] - g[3] - g[16] - g[17]);
    float Nz = 0.5f * (g[4] + g[14] + g[16] - g[5] - g[15] - g[17]);
    if (side == 0) {
        float rux = drho_b - (rest + 2.f * (g[1] + g[10] + g[11] + g[12] + g[13]));
        g[0] = g[1] + rux * (1.f / 3.f);
        g[6] = g[11] + rux * (1.f / 6.f) - Ny;
        g[7] = g[10] + rux * (1.f / 6.f) + Ny;
        g[8] = g[13] + rux * (1.f / 6.f) - Nz;
        g[9] = g[12] + rux * (1.f / 6.f) + Nz;
    } else {
        float rux = (rest + 2.f * (g[0] + g[6] + g[7] + g[8] + g[9])) - drho_b;
        g[1] = g[0] - rux * (1.f / 3.f);
        g[11] = g[6] - rux * (1.f / 6.f) + Ny;
        g[10] = g[7] - rux * (1.f / 6.f) - Ny;
        g[13] = g[8] - rux * (1.f / 6.f) + Nz;
        g[12] = g[9] - rux * (1.f / 6.f) - Nz;
    }
}

// Link lists for the link kernel.  Links are grouped by (sphere, direction
// m, maybe), each group padded to whole chunks of 32 records, and each
// sphere's groups together padded to whole LINK_WARP records, so a warp
// walks LINK_WARP / 32 chunks of one sphere, each chunk in one direction
// (one record per lane and chunk) and either without or with only `maybe`
// links:
//   warp_p[w]    = sphere index
//   chunk_dir[c] = direction m of chunk c (the solid neighbour is x + c_m),
//                  | 64 for a chunk of `maybe` links, | 128 when the chunk
//                  holds an `in_band` link; warp w owns chunks
//                  w LINK_CHUNKS ... (w + 1) LINK_CHUNKS - 1
//   link[r]      = {cidx of the fluid node x,
//                   (x - org) + 128 packed 8 bits per axis | maybe << 24 |
//                   shared << 25 | in_band << 26}
// `maybe` marks a neighbour inside a band: whether the sphere owns it now
// is decided by the map update's FP32 test (same operands and rounding),
// or by reading the owner map near the FP32 margin or when the band node
// has several candidate spheres (`shared`).  `in_band` marks a fluid node x
// that may itself be covered before the next re-layout (its fluid bit is
// read); every other link node stays fluid.  cidx == NONE pads.
constexpr int LINK_WARP = 256;
constexpr int LINK_CHUNKS = LINK_WARP / 32;  // chunks per warp
constexpr int LINK_GROUPS = 2 * (Q - 1);     // groups per sphere: (direction m, maybe) -> 2 m + maybe
static_assert(LINK_CHUNKS == 4 || LINK_CHUNKS == 8, "4 or 8 chunk directions per warp");

struct LinkLists {
    const uint2* link;
    const uint32_t* warp_p;
    const uint8_t* chunk_dir;  // LINK_CHUNKS bytes per warp
    uint32_t nwarps;
};

// Link word of a stored node, for the even steps' links inside the collide
// kernel (one 8-byte word per node):
//   .x = link mask (bit m, m < 18: the neighbour x + c_m is solid) | sphere A << 18
//   .y = B mask (bit m: that link's neighbour belongs to sphere B) | sphere B << 18
// Sphere indices take 14 bits; LW_NONE stands for no sphere B, and as sphere
// A for a node whose solid neighbours belong to more than two spheres (its
// links then read the owner map).  Built at the layout from the owner map
// and renewed for every converted node and its 18 neighbours.
constexpr uint32_t LW_MASK = (1u << 18) - 1u;
constexpr uint32_t LW_NONE = 0x3fffu;
constexpr int LW_MAX_SPHERES = (int)LW_NONE;  // sphere indices 0 .. LW_NONE - 1

// Nodes whose solid/fluid status can change before the next re-layout.
struct Band {
    const uint32_t* coord;  // packed x, y, z
    const int4* cand;       // up to 4 sphere indices, ascending, -1 padded
    const float* slack;     // distance to the nearest candidate surface at the layout (0: always re-test)
    uint32_t n;
};

struct Flip {
    uint32_t coord;
    int32_t old_owner, new_owner;
    uint32_t pad;
};

struct FlipBuf {
    Flip* rec;
    float* scratch;   // [cap][19][19]
    uint8_t* valid;   // [cap][19]
    uint32_t cap;
};

// DEM state (Section 2.2).
struct Dem {
    int n, K, cluster;
    float dt;                // 1 / K
    float kn, kt, mu;        // Eqs. 11-12 prefactors
    float3 g;                // body force
    int nbmax;
    // per particle
    const double* Xref;
    float4* dX;              // canonical displacement since re-layout
    float4* dXc;             // Kahan compensation
    float4* dXb;             // [2][n] double buffer read by the force phase
    float4* V;
    float4* W;
    float4* q;
    float4* Vhb;             // [2][n]
    float4* Whb;             // [2][n]
    float4* Fc;              // contact force (persistent across steps)
    float4* Tc;
    const double* Fh;        // hydrodynamic force/torque sums of this step (Eqs. 18-19)
    const double* Th;
    double* Fh_prev;         // the sums of the previous step
    double* Th_prev;
    float4* Fa;              // applied: mean of this and the previous step
    float4* Ta;
    const float* R;
    const float* invm;
    const float* invI;
    const uint8_t* fixed;
    // neighbour list
    const int* nb_cnt;
    const int* nb_j;
    const float4* nb_dref;   // xyz: X_ref_j + shift - X_ref_i, w: (R_i+R_j)^2 - |xyz|^2
    float4* nb_ft;           // tangential history (force on i)
    // outputs for the lattice kernels
    int4* org;
    int4* orgw;
    float4* xf;
    uint32_t* status;
    uint32_t* max_disp_bits;
    uint32_t* disp_layout_bits;
    uint32_t* layout_fresh;
    uint32_t* max_vel_bits;
    float hard_disp;             // displacement at which the layout is invalid
    int px;
    double Lx, Ly, Lz;
};

// lattice.cu
void launch_collide(const Lat& L, const Mon& mon, bool odd, bool monitor, int tile, cudaStream_t s);
void launch_collide_even_links(const Lat& L, const Mon& mon, const PartView& P, const uint2* lw, bool monitor,
                               int tile, cudaStream_t s);
void launch_inlet_outlet(const Lat& L, const BC& bc, bool after_even, cudaStream_t s);
void launch_plane_sums(const Lat& L, bool after_even, double* out, cudaStream_t s);
void launch_read_fields(const Lat& L, bool after_even, double* rho, double* u, uint8_t* solid,
                        cudaStream_t s);

// coupling.cu
void launch_links(const Lat& L, const PartView& P, const LinkLists& B, cudaStream_t s);
void launch_map_update(const Lat& L, const PartView& P, const Band& band, const FlipBuf& F,
                       DevStats* st, bool after_even, int step_parity, uint2* lw, bool shared_gpu,
                       cudaStream_t s);
void launch_link_words(const Lat& L, uint2* lw, cudaStream_t s);

// dem.cu
void launch_dem_step(const Dem& D, bool init_only, cudaStream_t s);
// adjoint.cu: reverse-mode kernels of the lattice step for a fixed packing
struct AdjArgs {
    Lat L;
    const uint32_t* nbr;  // [18][nSpad] compact index of x + c_m if fluid, else NONE
    float* adj;           // [19][nSpad] adjoint of the natural populations
    int inlet, outlet, probe_x;
};
void launch_adj_snapshot(const Lat& L, bool after_even, float* nat, cudaStream_t s);
void launch_adj_nbr(const Lat& L, uint32_t* nbr, cudaStream_t s);
void launch_adj_boundary(const AdjArgs& A, double shape, double* d_amp, cudaStream_t s);
void launch_adj_step(const AdjArgs& A, const float* nat, float* out, float dl, double* d_omega, cudaStream_t s);

// Parameter derivatives of the reverse kernels: each block sums its
// threads' terms and adds them to one of GRAD_COPIES FP64 accumulators
// (blockIdx % GRAD_COPIES: no long queue of atomics on one address); the
// host adds the copies.
constexpr int GRAD_COPIES = 64;
__device__ __forceinline__ void block_sum_to(double v, double* dst) {
    __shared__ double part[32];
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) part[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < (int)(blockDim.x >> 5) ? part[lane] : 0.0;
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && v != 0.0) atomicAdd(dst, v);
    }
}

// psm.cu: the smooth surrogate of the coupling (dense lattice) and its reverse
struct PsmArgs {
    int nx, ny, nz, px, inlet, outlet, probe_x;
    float rho_f, tau;
    size_t N;  // nodes
};
void launch_psm_eps(const PsmArgs& A, const double* X, const double* R, int n, float* eps, cudaStream_t s);
void launch_psm_step(const PsmArgs& A, const float* gin, float* gout, const float* eps, cudaStream_t s);
void launch_psm_boundary(const PsmArgs& A, float* g, const Source& src, unsigned long long t1, cudaStream_t s);
void launch_psm_probe(const PsmArgs& A, const float* g, double* out, cudaStream_t s);
void launch_psm_adj_boundary(const PsmArgs& A, float* lam, double shape, double* d_amp, cudaStream_t s);
void launch_psm_adj_step(const PsmArgs& A, const float* lin, const float* gt, float* lout, const float* eps, float dl,
                         double* d_tau, double* G, cudaStream_t s);
void launch_psm_grad_x(const PsmArgs& A, const double* G, const float* eps, const double* X, const double* R, int n,
                       double* dX, cudaStream_t s);
}  // namespace lbmdem
