// common.cuh -- lattice constants and the device-side views of the state.
//
// Compact lattice (the fluid is ~25% of the nodes in the FCC media, so a dense
// lattice that skips solids would still move ~2x the fluid bytes through
// partially used 32-byte sectors):
//   * S  = stored nodes = every node that is fluid now or within `skin` of a
//          sphere surface on the solid side (it may become fluid before the
//          next re-layout).  S = A + B, where A = nodes fluid at re-layout
//          time (lexicographic x, y, z order, indices [0, nA)) and B = the
//          remaining stored nodes (indices [nA, nS)), so the streamed region A
//          is dense in fluid and B is only touched where a node converted.
//   * f  = populations as deviations g_i = f_i - w_i rho_f, structure of
//          arrays [19][nSpad], in place with the AA access pattern; stored as
//          FP32, or as BF16 / FP16 scaled by a power of two (FP16: 2^12, so
//          that deviations of 1e-8 .. 16 stay normal numbers), always
//          collided in FP32.
//   * rec[w] = {maskF, maskA, baseA, baseB} for every 32-node word of a
//          z-line: fluid-now bits, region-A bits and the compact indices of the
//          first A and B node of the word; maskB[w] holds the B bits.  The
//          compact index of a stored node is base + popc(mask & lower bits).
//          The word table (16 B per 32 nodes) stays resident in L2.
//   * coord[i] = x << 20 | y << 10 | z of compact node i.
//   * fbits[i / 32] = fluid-now bit of compact node i.
//   * owner[lattice index] = index of the sphere a node belongs to, or FLUID.
//
// AA pattern, with fluid-solid links handled in place (Section 2.3):
//   even step: node x reads slot m of itself, writes post-collision value of
//              direction m into slot opp(m) of itself;
//   odd step:  node x reads direction m from slot opp(m) of x - c_m when that
//              node is fluid, else from slot m of x itself; it writes
//              direction m into slot m of x + c_m when fluid, else into slot
//              opp(m) of x itself.
//   After either step, slot opp(d) of a fluid node x whose neighbour x + c_d
//   is solid holds the post-collision value of direction d; the link kernel
//   turns it into the bounced value (Eq. 14) in place.  Populations arriving
//   from outside the x range are treated the same way (resting wall) before
//   the inlet/outlet overwrite them.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbmdem {

constexpr int Q = 19;
constexpr int32_t OWNER_FLUID = 0x7fffffff;
constexpr uint32_t NONE = 0xffffffffu;

// D3Q19 velocities in the column order of Eq. 3 (index m = d - 1).
__host__ __device__ constexpr int cx(int m) {
    return (m == 0 || m == 6 || m == 7 || m == 8 || m == 9) ? 1
           : (m == 1 || m == 10 || m == 11 || m == 12 || m == 13) ? -1
                                                                  : 0;
}
__host__ __device__ constexpr int cy(int m) {
    return (m == 2 || m == 6 || m == 10 || m == 14 || m == 15) ? 1
           : (m == 3 || m == 7 || m == 11 || m == 16 || m == 17) ? -1
                                                                 : 0;
}
__host__ __device__ constexpr int cz(int m) {
    return (m == 4 || m == 8 || m == 12 || m == 14 || m == 16) ? 1
           : (m == 5 || m == 9 || m == 13 || m == 15 || m == 17) ? -1
                                                                 : 0;
}
// Eq. 8 weights by speed class.
__host__ __device__ constexpr float wt(int m) {
    return (cx(m) * cx(m) + cy(m) * cy(m) + cz(m) * cz(m)) == 0 ? 1.0f / 3.0f
           : (cx(m) * cx(m) + cy(m) * cy(m) + cz(m) * cz(m)) == 1 ? 1.0f / 18.0f
                                                                  : 1.0f / 36.0f;
}
// Opposite direction: the pairs of Eq. 3 are (0,1) (2,3) (4,5) (6,11) (7,10)
// (8,13) (9,12) (14,17) (15,16) and 18 alone.
__host__ __device__ constexpr int opp(int m) {
    return m == 18 ? 18
           : m < 6 ? (m ^ 1)
           : m == 6 ? 11
           : m == 11 ? 6
           : m == 7 ? 10
           : m == 10 ? 7
           : m == 8 ? 13
           : m == 13 ? 8
           : m == 9 ? 12
           : m == 12 ? 9
           : m == 14 ? 17
           : m == 17 ? 14
           : m == 15 ? 16
                     : 15;
}

__host__ __device__ inline uint32_t pack_coord(int x, int y, int z) {
    return ((uint32_t)x << 20) | ((uint32_t)y << 10) | (uint32_t)z;
}
__host__ __device__ inline void unpack_coord(uint32_t c, int& x, int& y, int& z) {
    x = (int)(c >> 20);
    y = (int)((c >> 10) & 1023u);
    z = (int)(c & 1023u);
}

// Lattice geometry and the compact-storage views, passed by value.
struct Lat {
    int nx, ny, nz, nw;   // nw = 32-node words per z-line
    int px;               // x periodic
    uint32_t nA, nS, nSpad;
    void* f;              // [19][nSpad] deviations, element type by `st`
    int st;               // storage: 0 FP32, 1 BF16, 2 FP16 (scaled by fs)
    float fs, fsi;        // storage scale and its inverse (powers of two)
    uint4* rec;           // [nx*ny*nw] {maskF, maskA, baseA, baseB}
    uint32_t* maskB;      // [nx*ny*nw]
    uint32_t* coord;      // [nSpad]
    uint32_t* fbits;      // [nSpad / 32]
    int32_t* owner;       // [nx*ny*nz]
    float tau_inv;
    float rho_f;
};

__device__ __forceinline__ int wrap1(int a, int L) { return a < 0 ? a + L : (a >= L ? a - L : a); }

// minimum image of an offset -L < d < L
__device__ __forceinline__ int imin_small(int d, int L) {
    if (2 * d > L) return d - L;
    if (2 * d < -L) return d + L;
    return d;
}

// Compact index of node (x+dx, y+dy, z+dz) if it is fluid now, else NONE.
// dx, dy, dz in {-1, 0, 1}.  Out-of-range x (non-periodic) returns NONE.
__device__ __forceinline__ uint32_t fluid_index(const Lat& L, int x, int y, int z, int dx, int dy,
                                                int dz) {
    int xs = x + dx;
    if (L.px) {
        xs = wrap1(xs, L.nx);
    } else if (xs < 0 || xs >= L.nx) {
        return NONE;
    }
    int ys = wrap1(y + dy, L.ny), zs = wrap1(z + dz, L.nz);
    uint32_t wi = ((uint32_t)xs * L.ny + ys) * L.nw + (zs >> 5);
    uint4 r = __ldg(&L.rec[wi]);
    uint32_t bit = 1u << (zs & 31);
    if (!(r.x & bit)) return NONE;
    uint32_t low = bit - 1u;
    if (r.y & bit) return r.z + __popc(r.y & low);
    return r.w + __popc(__ldg(&L.maskB[wi]) & low);
}

// Same for a node given directly (used outside the hot kernel; reads the
// record with a coherent load because the map-update kernels modify it).
__device__ __forceinline__ uint32_t stored_index(const Lat& L, int x, int y, int z, bool& fluid) {
    uint32_t wi = ((uint32_t)x * L.ny + y) * L.nw + (z >> 5);
    uint4 r = L.rec[wi];
    uint32_t bit = 1u << (z & 31);
    fluid = (r.x & bit) != 0;
    uint32_t low = bit - 1u;
    if (r.y & bit) return r.z + __popc(r.y & low);
    uint32_t mb = L.maskB[wi];
    if (mb & bit) return r.w + __popc(mb & low);
    return NONE;
}

__device__ __forceinline__ bool fluid_bit(const Lat& L, uint32_t i) {
    return (L.fbits[i >> 5] >> (i & 31)) & 1u;
}

// Population storage types and their FP32 conversions (round to nearest;
// the scale is a power of two, so scaling is exact).
template <int ST> struct PopT;
template <> struct PopT<0> { using T = float; };
template <> struct PopT<1> { using T = __nv_bfloat16; };
template <> struct PopT<2> { using T = __half; };

template <int ST> __device__ __forceinline__ float to_f(typename PopT<ST>::T v, float fsi);
template <> __device__ __forceinline__ float to_f<0>(float v, float) { return v; }
template <> __device__ __forceinline__ float to_f<1>(__nv_bfloat16 v, float fsi) { return __bfloat162float(v) * fsi; }
template <> __device__ __forceinline__ float to_f<2>(__half v, float fsi) { return __half2float(v) * fsi; }

template <int ST> __device__ __forceinline__ typename PopT<ST>::T from_f(float v, float fs);
template <> __device__ __forceinline__ float from_f<0>(float v, float) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<1>(float v, float fs) { return __float2bfloat16_rn(v * fs); }
template <> __device__ __forceinline__ __half from_f<2>(float v, float fs) { return __float2half_rn(v * fs); }

template <int ST> __device__ __forceinline__ typename PopT<ST>::T* pops(const Lat& L) {
    return static_cast<typename PopT<ST>::T*>(L.f);
}

// Location of population m of fluid node (x,y,z) with compact index i, in the
// state between steps.  after_even = true: the state after an even step
// (natural populations sit in the neighbours' reversed slots).
template <int ST>
__device__ __forceinline__ typename PopT<ST>::T* pop_loc(const Lat& L, bool after_even, int x, int y, int z,
                                                         uint32_t i, int m) {
    typename PopT<ST>::T* f = pops<ST>(L);
    if (!after_even || m == 18) return f + (size_t)m * L.nSpad + i;
    uint32_t s = fluid_index(L, x, y, z, -cx(m), -cy(m), -cz(m));
    if (s == NONE) return f + (size_t)m * L.nSpad + i;
    return f + (size_t)opp(m) * L.nSpad + s;
}

// Particles as seen by the lattice kernels (current time level).
struct PartView {
    int n;
    const double* Xref;   // [n][3] reference centres of the current layout
    const float4* dX;     // [n] displacement since re-layout (xyz), w unused
    const float4* dXc;    // [n] Kahan compensation of dX
    const float4* V;      // [n]
    const float4* W;      // [n]
    const float* R;       // [n]
    const double* Rd;     // [n] radii in FP64 for the exact inside test
    const int4* org;      // [n] integer origin floor(Xref)
    const int4* orgw;     // [n] that origin wrapped into the box (periodic axes)
    const float4* xf;     // [n] X(t) - origin, FP32
    float4* ab;           // [n][Q-1] moving-wall terms of the step's links (alpha - xf.beta, beta)
    float4* pk;           // [n][3] sphere packet of the step: {xf, V.x} {V.y, V.z, W.x, W.y}
                          // {W.z, wrapped origin as int bits}
    double* Fh;           // [NREP][n][3] hydrodynamic force accumulators (summed by the DEM)
    double* Th;           // [NREP][n][3] hydrodynamic torque accumulators
};

// The link kernel spreads its atomics over NREP copies of each sphere's
// force and torque accumulators (fewer same-address collisions); the DEM
// kernel and the read-out sum the copies.
constexpr int NREP = 4;

// Exact "inside" test shared by painting and the map update: |y - X|^2 < R^2
// in FP64 without contraction, X = Xref + dX (+ compensation).
__device__ __forceinline__ bool inside_exact(double ax, double ay, double az, double R) {
    double s = __dadd_rn(__dadd_rn(__dmul_rn(ax, ax), __dmul_rn(ay, ay)), __dmul_rn(az, az));
    return s < __dmul_rn(R, R);
}

// FP32 |a|^2 with a fixed rounding (no contraction), used identically by the
// map update and the link kernel so that both take the same decisions.
__device__ __forceinline__ float norm2_rn(float ax, float ay, float az) {
    return __fadd_rn(__fadd_rn(__fmul_rn(ax, ax), __fmul_rn(ay, ay)), __fmul_rn(az, az));
}
// the FP32 inside test decides only outside this relative margin of R^2
constexpr float FP32_MARGIN = 1e-5f;

// |y - X|^2 / R^2 with the same operation order and rounding as the test
// above; among the spheres that contain a node, the smallest ratio owns it.
__device__ __forceinline__ double inside_ratio(double ax, double ay, double az, double R) {
    double s = __dadd_rn(__dadd_rn(__dmul_rn(ax, ax), __dmul_rn(ay, ay)), __dmul_rn(az, az));
    return __ddiv_rn(s, __dmul_rn(R, R));
}

__device__ __forceinline__ double minimg(double d, double L, int periodic) {
    if (!periodic) return d;
    return d - L * floor(d / L + 0.5);
}

// Device status bits (latched; host maps them to LBMDEM_ERR_*).
enum : uint32_t {
    ST_UNSTABLE = 1u,
    ST_CAPACITY = 2u,
    ST_SKIN = 4u,
    ST_TIMEOUT = 8u,
};

struct DevStats {
    uint32_t status;
    uint32_t nflip[2];    // conversions queued this step (double-buffered by step parity)
    uint32_t max_disp_bits;  // float bits of max |dX| (non-negative)
    uint32_t max_vel_bits;   // float bits of max |V|
    uint32_t disp_layout_bits;  // float bits of max |dX| seen since the layout build
    unsigned long long t;    // steps begun (the map update counts each step first; between
                             // steps it equals the completed steps)
    unsigned long long flips_total;
    double mon[6];           // sum rho, sum rho u, max|u|, step
    uint32_t max_u_bits;
    uint32_t layout_fresh;   // 1 from a layout build until the first step's DEM
};

// Programmatic dependent launch.  The kernels of a step are launched with
// programmatic stream serialization (launch_pdl): such a kernel may be
// scheduled while its predecessor on the stream is still running, and its
// first statement, pdl_wait(), blocks until the predecessor grid has
// completed and its memory operations are visible, so nothing is read or
// written early.  pdl_trigger() in the predecessor lets the successor launch
// once every block of the predecessor has executed it (blocks that exit
// count as triggered), which hides the successor's launch and block
// scheduling behind the predecessor's tail.  Both are no-ops for a kernel
// launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*k)(KArgs...), unsigned grid, unsigned block, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(block, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

}  // namespace lbmdem
