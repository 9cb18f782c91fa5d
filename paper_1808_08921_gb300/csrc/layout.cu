// layout.cu -- building the compact lattice from the sphere positions.
//
// Run at set_packing and at every re-layout (when some sphere has moved a
// good part of the skin since the last one).  Steps:
//   1. paint: for every sphere, every node within R + skin of its centre
//      (all periodic images; the box's lines visit only that ball) is
//      tested with the exact FP64 rule |y - X|^2 < R^2 shared with
//      the map update; a node inside several spheres belongs to the one with
//      the smallest |y - X|^2 / R^2 (first pass: atomicMin of the FP64 ratio
//      bits; second pass: lowest index among the equal ratios).
//      Only set_packing paints owners: after step t the map belongs to the
//      positions of that step's map update, one DEM update behind the
//      current ones, so a re-layout keeps the maintained map (the next map
//      update converts what the newer positions cover or uncover).
//      Nodes deeper than `skin` inside a sphere are flagged "deep" (never
//      stored); nodes within `skin` of a surface are flagged "band" (re-tested
//      every step).  The inlet/outlet planes are never solid.
//   2. word masks and counts per 32-node word; exclusive scans give the
//      compact indices (region A = fluid now, region B = stored solid).
//   3. compact coordinates, fluid bits, band list with candidate spheres,
//      per-sphere surface lists for the link kernel (warp-padded; the box's
//      lines visit only the shell where link nodes can be), and, on a
//      re-layout, the populations copied from the old compact order.
#include "common.cuh"
#include "kernels.cuh"
#include "layout.cuh"

namespace lbmdem {

__global__ void k_fill_i32(int32_t* p, int32_t v, size_t n) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

void fill_i32(int32_t* p, int32_t v, size_t n, cudaStream_t s) {
    if (n) k_fill_i32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, v, n);
}

// ------------------------------------------------------------ scan

// exclusive scan of 1024-element tiles (256 threads x 4), tile sums out
__global__ void k_scan_tile(const uint32_t* in, uint32_t* out, uint32_t* sums, size_t n) {
    __shared__ uint32_t sh[256];
    size_t base = (size_t)blockIdx.x * 1024;
    uint32_t v[4];
    uint32_t tot = 0;
    for (int k = 0; k < 4; ++k) {
        size_t i = base + threadIdx.x * 4 + k;
        v[k] = i < n ? in[i] : 0u;
        tot += v[k];
    }
    sh[threadIdx.x] = tot;
    __syncthreads();
    for (int o = 1; o < 256; o <<= 1) {
        uint32_t a = threadIdx.x >= (unsigned)o ? sh[threadIdx.x - o] : 0u;
        __syncthreads();
        sh[threadIdx.x] += a;
        __syncthreads();
    }
    uint32_t run = sh[threadIdx.x] - tot;
    for (int k = 0; k < 4; ++k) {
        size_t i = base + threadIdx.x * 4 + k;
        if (i < n) out[i] = run;
        run += v[k];
    }
    if (threadIdx.x == 255) sums[blockIdx.x] = sh[255];
}

__global__ void k_scan_add(uint32_t* out, const uint32_t* sums, size_t n) {
    size_t i = (size_t)blockIdx.x * 1024 + threadIdx.x * 4;
    uint32_t a = sums[blockIdx.x];
    for (int k = 0; k < 4; ++k)
        if (i + k < n) out[i + k] += a;
}

// out = exclusive scan of in (may alias); tmp needs scan_tmp_size(n) words.
void exclusive_scan(const uint32_t* in, uint32_t* out, size_t n, uint32_t* tmp, cudaStream_t s) {
    if (n == 0) return;
    size_t tiles = (n + 1023) / 1024;
    uint32_t* sums = tmp;
    k_scan_tile<<<(unsigned)tiles, 256, 0, s>>>(in, out, sums, n);
    if (tiles > 1) {
        exclusive_scan(sums, sums, tiles, tmp + tiles, s);
        k_scan_add<<<(unsigned)tiles, 256, 0, s>>>(out, sums, n);
    }
}

size_t scan_tmp_size(size_t n) {
    size_t t = 0;
    while (n > 1) {
        n = (n + 1023) / 1024;
        t += n;
    }
    return t + 1;
}

// ------------------------------------------------------------ box lines

__device__ __forceinline__ int wrapi(int a, int L) {
    int r = a % L;
    return r < 0 ? r + L : r;
}

// The nodes of a sphere's box [x0, x0 + ex) x [y0, y0 + ey) x [z0, z1] that
// a kernel has to visit: on each line (x, y) at most two z-intervals
// [a0, a1] and [b0, b1] (empty when lo > hi), given by the caller from the
// line's distance to the centre; the rest of the box is known to need
// nothing.  One thread block per sphere (BOX_THREADS threads): lines are
// taken BOX_THREADS at a time, a block scan places their nodes, and each
// round gives every thread one node in (x, y, z) order -- the order of the
// whole-box loop with the skipped nodes left out.  Every thread calls
// `body(valid, x, y, z)` in every round (valid false past the last node), so
// the body may synchronise the block.
constexpr int BOX_THREADS = 256;

struct LineSpan {
    int a0, a1, b0, b1;
};

struct BoxLines {
    int x0, y0, z0, z1, ex, ey;
};

// the nodes with |z - zc| <= a, minus those with |z - zc| < b (b <= 0: none
// removed), within [z0, z1]
__device__ __forceinline__ LineSpan line_span(double zc, double a2, double b2, int z0, int z1) {
    LineSpan s = {0, -1, 0, -1};
    if (!(a2 >= 0.0)) return s;
    const double a = sqrt(a2);
    const int lo = max(z0, (int)ceil(zc - a)), hi = min(z1, (int)floor(zc + a));
    if (lo > hi) return s;
    s.a0 = lo;
    s.a1 = hi;
    if (b2 > 0.0) {
        const double b = sqrt(b2);
        const int e0 = (int)floor(zc - b) + 1, e1 = (int)ceil(zc + b) - 1;  // strictly inside
        if (e0 <= e1) {
            s.a1 = min(hi, e0 - 1);
            s.b0 = max(lo, e1 + 1);
            s.b1 = hi;
        }
    }
    return s;
}

template <class SpanFn, class Body>
__device__ void for_box_nodes(const BoxLines& B, SpanFn span, Body body) {
    __shared__ int s_a0[BOX_THREADS], s_la[BOX_THREADS], s_b0[BOX_THREADS];
    __shared__ uint32_t s_start[BOX_THREADS + 1];
    const uint32_t tid = threadIdx.x, nt = blockDim.x;
    const uint32_t nlines = (uint32_t)B.ex * (uint32_t)B.ey;
    for (uint32_t l0 = 0; l0 < nlines; l0 += nt) {
        LineSpan sp = {0, -1, 0, -1};
        if (l0 + tid < nlines) sp = span(B.x0 + (int)((l0 + tid) / (uint32_t)B.ey), B.y0 + (int)((l0 + tid) % (uint32_t)B.ey));
        const int la = max(sp.a1 - sp.a0 + 1, 0), lb = max(sp.b1 - sp.b0 + 1, 0);
        s_a0[tid] = sp.a0;
        s_la[tid] = la;
        s_b0[tid] = sp.b0;
        s_start[tid + 1] = (uint32_t)(la + lb);
        if (tid == 0) s_start[0] = 0u;
        __syncthreads();
        for (uint32_t o = 1; o < nt; o <<= 1) {  // inclusive scan of the counts
            const uint32_t v = tid >= o ? s_start[tid + 1 - o] : 0u;
            __syncthreads();
            s_start[tid + 1] += v;
            __syncthreads();
        }
        const uint32_t total = s_start[nt];
        for (uint32_t c0 = 0; c0 < total; c0 += nt) {
            const uint32_t c = c0 + tid;
            const bool valid = c < total;
            int xi = 0, yi = 0, zi = 0;
            if (valid) {
                uint32_t lo = 0, hi = nt;  // s_start[lo] <= c < s_start[hi]
                while (hi - lo > 1) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (s_start[mid] <= c) lo = mid;
                    else hi = mid;
                }
                const int o = (int)(c - s_start[lo]);
                zi = o < s_la[lo] ? s_a0[lo] + o : s_b0[lo] + (o - s_la[lo]);
                xi = B.x0 + (int)((l0 + lo) / (uint32_t)B.ey);
                yi = B.y0 + (int)((l0 + lo) % (uint32_t)B.ey);
            }
            body(valid, xi, yi, zi);
        }
        __syncthreads();  // the next batch rewrites the spans
    }
}

// ------------------------------------------------------------ painting

// Nodes farther than R + skin from the centre are left alone (neither
// owned, deep nor band), so each line visits |z - Z| <= sqrt((R + skin +
// 0.01)^2 - rho^2) only.
template <int PASS>
__global__ void __launch_bounds__(BOX_THREADS) k_paint(PaintArgs A) {
    const int p = blockIdx.x;
    const double X0 = A.X[3 * p], X1 = A.X[3 * p + 1], X2 = A.X[3 * p + 2];
    const double R = A.R[p];
    const double reach = R + A.skin + 1.0;
    BoxLines B;
    B.x0 = (int)ceil(X0 - reach);
    B.y0 = (int)ceil(X1 - reach);
    B.z0 = (int)ceil(X2 - reach);
    B.z1 = (int)floor(X2 + reach);
    B.ex = (int)floor(X0 + reach) - B.x0 + 1;
    B.ey = (int)floor(X1 + reach) - B.y0 + 1;
    const double Rin = R - A.skin, Rout = R + A.skin;
    const double rv = Rout + 0.01;
    auto span = [&](int xi, int yi) {
        const double ax = (double)xi - X0, ay = (double)yi - X1;
        return line_span(X2, rv * rv - (ax * ax + ay * ay), 0.0, B.z0, B.z1);
    };
    for_box_nodes(B, span, [&](bool valid, int xi, int yi, int zi) {
        if (!valid) return;
        int x;
        if (A.px) {
            x = wrapi(xi, A.nx);
        } else {
            if (xi <= 0 || xi >= A.nx - 1) return;  // boundary planes stay fluid
            x = xi;
        }
        const int y = wrapi(yi, A.ny), z = wrapi(zi, A.nz);
        const double ax = (double)xi - X0, ay = (double)yi - X1, az = (double)zi - X2;
        const size_t li = ((size_t)x * A.ny + y) * A.nz + z;
        if (A.owner && inside_exact(ax, ay, az, R)) {
            unsigned long long rb = (unsigned long long)__double_as_longlong(inside_ratio(ax, ay, az, R));
            if (PASS == 0)
                atomicMin(&A.best[li], rb);
            else if (A.best[li] == rb)
                atomicMin(&A.owner[li], p);
        }
        if (PASS == 1) return;
        const double d2 = ax * ax + ay * ay + az * az;
        if (Rin > 0 && d2 < Rin * Rin) A.deep[li] = 1;
        if (d2 < Rout * Rout && (Rin <= 0 || d2 >= Rin * Rin)) A.band[li] = 1;
    });
}

// word masks: maskF = maskA = stored fluid, maskB = stored solid
__global__ void k_words(LayoutArgs A) {
    size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t W = (size_t)A.nx * A.ny * A.nw;
    if (w >= W) return;
    int wz = (int)(w % A.nw);
    size_t line = w / A.nw;
    uint32_t mA = 0, mB = 0;
    for (int b = 0; b < 32; ++b) {
        int z = wz * 32 + b;
        if (z >= A.nz) break;
        size_t li = line * A.nz + z;
        bool fluid = A.owner[li] == OWNER_FLUID;
        if (A.deep[li] && !fluid) continue;
        if (fluid)
            mA |= 1u << b;
        else
            mB |= 1u << b;
    }
    A.rec[w] = make_uint4(mA, mA, 0u, 0u);
    A.maskB[w] = mB;
    A.cntA[w] = __popc(mA);
    A.cntB[w] = __popc(mB);
}

__global__ void k_words_bases(LayoutArgs A, uint32_t nA) {
    size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t W = (size_t)A.nx * A.ny * A.nw;
    if (w >= W) return;
    A.rec[w].z = A.cntA[w];
    A.rec[w].w = nA + A.cntB[w];
}

__global__ void k_coords(LayoutArgs A) {
    size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t W = (size_t)A.nx * A.ny * A.nw;
    if (w >= W) return;
    int wz = (int)(w % A.nw);
    size_t line = w / A.nw;
    int y = (int)(line % A.ny), x = (int)(line / A.ny);
    uint4 r = A.rec[w];
    uint32_t mB = A.maskB[w];
    uint32_t ia = r.z, ib = r.w;
    for (int b = 0; b < 32; ++b) {
        uint32_t bit = 1u << b;
        int z = wz * 32 + b;
        if (r.y & bit) A.coord[ia++] = pack_coord(x, y, z);
        if (mB & bit) A.coord[ib++] = pack_coord(x, y, z);
    }
}

__global__ void k_fbits(uint32_t* fbits, uint32_t nA, uint32_t nwords) {
    uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nwords) return;
    uint32_t lo = k * 32;
    uint32_t v;
    if (lo + 32 <= nA) v = 0xffffffffu;
    else if (lo >= nA) v = 0u;
    else v = (1u << (nA - lo)) - 1u;
    fbits[k] = v;
}

// re-layout: copy the natural populations (state between an odd and an even
// step: population m of node i sits in slot m of i) into the new order
template <typename T>
__global__ void k_gather_old(Lat Lnew, Lat Lold) {
    T* fn = static_cast<T*>(Lnew.f);
    const T* fo = static_cast<const T*>(Lold.f);
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Lnew.nA) return;
    int x, y, z;
    unpack_coord(Lnew.coord[i], x, y, z);
    bool fl;
    uint32_t o = stored_index(Lold, x, y, z, fl);
    if (o == NONE) return;
#pragma unroll
    for (int m = 0; m < Q; ++m) fn[(size_t)m * Lnew.nSpad + i] = fo[(size_t)m * Lold.nSpad + o];
}

// band nodes: compact list of (coord) via atomics; candidates found later
__global__ void k_band_collect(LayoutArgs A, uint32_t* band_coord, uint32_t* count, uint32_t cap) {
    size_t li = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t N = (size_t)A.nx * A.ny * A.nz;
    if (li >= N || !A.band[li]) return;
    int z = (int)(li % A.nz);
    size_t r = li / A.nz;
    int y = (int)(r % A.ny), x = (int)(r / A.ny);
    uint32_t k = atomicAdd(count, 1u);
    if (k < cap) band_coord[k] = pack_coord(x, y, z);
}

// link lists: for every stored node x within R + skin + 1.5 of a sphere and
// every direction m, a link if x + c_m is owned by the sphere and outside
// every band (fixed until the next re-layout), or a `maybe` link if x + c_m
// is a band node within R + skin of the sphere (owner read each step).  A
// link node x that is itself in a band carries `in_band` (its fluid bit is
// read each step).
struct SurfNode {
    uint32_t ci;
    int ox, oy, oz;           // x - floor(Xref)
    uint32_t sure, maybe, shared;
    bool in_band;
};

// The geometry is FP32 (FP64 arithmetic is slow on this part): the offset
// from the centre is formed in FP64 and rounded once (|offset| < 2 reach),
// and both tests carry a relative margin of 1e-5 on squared distances, far
// above FP32 rounding: the reach test only has to keep a superset of the
// link nodes, and the image test separates distances below R (owned) from
// distances above L - R - skin (another image), both at least the skin away
// from R + skin.
__device__ __forceinline__ bool surf_node(const SurfArgs& A, int p, int xi, int yi, int zi, SurfNode& sn) {
    int x;
    if (A.L.px) x = wrapi(xi, A.L.nx);
    else {
        if (xi < 0 || xi >= A.L.nx) return false;
        x = xi;
    }
    int y = wrapi(yi, A.L.ny), z = wrapi(zi, A.L.nz);
    const double X0 = A.X[3 * p], X1 = A.X[3 * p + 1], X2 = A.X[3 * p + 2];
    const float ax = (float)((double)xi - X0), ay = (float)((double)yi - X1), az = (float)((double)zi - X2);
    const float Rp = (float)A.R[p];
    const float reach = Rp + (float)A.reach_extra;
    if (ax * ax + ay * ay + az * az >= reach * reach * (1.0f + 1e-5f)) return false;
    bool fl;
    uint32_t ci = stored_index(A.L, x, y, z, fl);
    if (ci == NONE) return false;
    const bool in_band = A.band[((size_t)x * A.L.ny + y) * A.L.nz + z] != 0;
    const float Rb2 = (Rp + (float)A.skin) * (Rp + (float)A.skin) * (1.0f + 1e-5f);
    uint32_t sure = 0, maybe = 0, shared = 0;
#pragma unroll
    for (int m = 0; m < Q - 1; ++m) {
        int xs = x + cx(m);
        if (A.L.px) xs = wrapi(xs, A.L.nx);
        else if (xs < 0 || xs >= A.L.nx) continue;
        int ys = wrapi(y + cy(m), A.L.ny), zs = wrapi(z + cz(m), A.L.nz);
        size_t li = ((size_t)xs * A.L.ny + ys) * A.L.nz + zs;
        // the neighbour's offset from the centre in this visit's image: a
        // periodic axis narrower than 2 (R + skin + 1.5) brings a node near
        // two images of one sphere, and each of its links belongs to the
        // image whose R + skin contains the neighbour (R + skin < L / 2
        // makes that image unique), with that image's lever
        const float bx = ax + (float)cx(m), by = ay + (float)cy(m), bz = az + (float)cz(m);
        const bool this_image = bx * bx + by * by + bz * bz < Rb2;
        if (A.band[li]) {
            if (this_image) {
                maybe |= 1u << m;
                if (A.band[li] >= 2) shared |= 1u << m;
            }
        } else if (A.owner[li] == p && this_image) {
            sure |= 1u << m;
        }
    }
    if (!(sure | maybe)) return false;
    sn.ci = ci;
    sn.ox = xi - (int)floor(X0);
    sn.oy = yi - (int)floor(X1);
    sn.oz = zi - (int)floor(X2);
    sn.sure = sure;
    sn.maybe = maybe;
    sn.shared = shared;
    sn.in_band = in_band;
    return true;
}

// The candidates of sphere p's surface lists: the box of the reach test,
// line by line from the inner radius R - skin - 0.01 (deeper nodes are
// never stored, except on the non-periodic boundary planes, which are
// never deep) to the reach test's radius with a relative margin of 1e-4
// over its FP32 rounding.  surf_node() still decides every candidate, so the
// lists are those of the whole box, in the same order.
__device__ __forceinline__ BoxLines surf_box(const SurfArgs& A, int p) {
    const double reach = A.R[p] + A.reach_extra;
    BoxLines B;
    B.x0 = (int)ceil(A.X[3 * p] - reach);
    B.y0 = (int)ceil(A.X[3 * p + 1] - reach);
    B.z0 = (int)ceil(A.X[3 * p + 2] - reach);
    B.z1 = (int)floor(A.X[3 * p + 2] + reach);
    B.ex = (int)floor(A.X[3 * p] + reach) - B.x0 + 1;
    B.ey = (int)floor(A.X[3 * p + 1] + reach) - B.y0 + 1;
    return B;
}

__device__ __forceinline__ LineSpan surf_span(const SurfArgs& A, int p, int xi, int yi, int z0, int z1) {
    const double X0 = A.X[3 * p], X1 = A.X[3 * p + 1], X2 = A.X[3 * p + 2];
    const double reach = (double)((float)A.R[p] + (float)A.reach_extra);
    const double ax = (double)xi - X0, ay = (double)yi - X1, rho2 = ax * ax + ay * ay;
    const double rin = A.R[p] - A.skin - 0.01;
    const bool plane = !A.L.px && (xi == 0 || xi == A.L.nx - 1);
    const double b2 = rin > 0.0 && !plane ? rin * rin - rho2 : 0.0;
    return line_span(X2, reach * reach * (1.0 + 1e-4) + 0.05 - rho2, b2, z0, z1);
}

// per sphere: links per direction, padded to whole 32-record chunks; the
// sphere's total is padded to whole LINK_WARP groups on its last direction
__global__ void __launch_bounds__(BOX_THREADS) k_surf_count(SurfArgs A) {
    const int p = blockIdx.x;
    const BoxLines B = surf_box(A, p);
    __shared__ uint32_t cnt[LINK_GROUPS];
    if (threadIdx.x < LINK_GROUPS) cnt[threadIdx.x] = 0;
    __syncthreads();
    for_box_nodes(B, [&](int xi, int yi) { return surf_span(A, p, xi, yi, B.z0, B.z1); },
                  [&](bool valid, int xi, int yi, int zi) {
                      SurfNode sn;
                      if (!valid || !surf_node(A, p, xi, yi, zi, sn)) return;
                      for (int m = 0; m < Q - 1; ++m) {
                          if (sn.sure >> m & 1u) atomicAdd(&cnt[2 * m], 1u);
                          if (sn.maybe >> m & 1u) atomicAdd(&cnt[2 * m + 1], 1u);
                      }
                  });
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t tot = 0, raw = 0;
        for (int g = 0; g < LINK_GROUPS; ++g) {
            raw += cnt[g];
            cnt[g] = (cnt[g] + 31u) / 32u * 32u;
            tot += cnt[g];
        }
        atomicAdd(A.nlink, raw);
        cnt[LINK_GROUPS - 1] += (tot + (LINK_WARP - 1)) / LINK_WARP * LINK_WARP - tot;
    }
    __syncthreads();
    if (threadIdx.x < LINK_GROUPS) A.count[(size_t)p * LINK_GROUPS + threadIdx.x] = cnt[threadIdx.x];
}

// fill in a deterministic order: per direction, rounds of blockDim
// candidates in bounding-box order, block prefix sums over the round
__global__ void __launch_bounds__(BOX_THREADS) k_surf_fill(SurfArgs A) {
    const int p = blockIdx.x;
    const BoxLines B = surf_box(A, p);
    __shared__ uint32_t sh[LINK_GROUPS][33];
    __shared__ uint32_t run[LINK_GROUPS];
    if (threadIdx.x < LINK_GROUPS) run[threadIdx.x] = 0;
    __syncthreads();
    uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for_box_nodes(B, [&](int xi, int yi) { return surf_span(A, p, xi, yi, B.z0, B.z1); },
                  [&](bool valid, int xi, int yi, int zi) {
        SurfNode sn;
        bool ok = valid && surf_node(A, p, xi, yi, zi, sn);
        // group 2 m + 1 takes the `maybe` links of direction m, 2 m the others
        uint32_t sure = ok ? sn.sure : 0u, maybe = ok ? sn.maybe : 0u;
        for (int g = 0; g < LINK_GROUPS; ++g) {
            unsigned bal = __ballot_sync(0xffffffffu, (((g & 1) ? maybe : sure) >> (g >> 1)) & 1u);
            if (lane == 0) sh[g][wid] = __popc(bal);
        }
        __syncthreads();
        if (threadIdx.x < LINK_GROUPS) {
            uint32_t s = 0;
            for (uint32_t k = 0; k < nwarp; ++k) {
                uint32_t c = sh[threadIdx.x][k];
                sh[threadIdx.x][k] = s;
                s += c;
            }
            sh[threadIdx.x][32] = s;
        }
        __syncthreads();
        uint32_t rel = ok ? ((uint32_t)(sn.ox + 128) | ((uint32_t)(sn.oy + 128) << 8) |
                             ((uint32_t)(sn.oz + 128) << 16))
                          : 0u;
        for (int g = 0; g < LINK_GROUPS; ++g) {
            const int m = g >> 1;
            const bool mine = (((g & 1) ? maybe : sure) >> m) & 1u;
            unsigned bal = __ballot_sync(0xffffffffu, mine);
            if (!mine) continue;
            uint32_t before = __popc(bal & ((1u << lane) - 1u));
            uint32_t pos = A.offset[(size_t)p * LINK_GROUPS + g] + run[g] + sh[g][wid] + before;
            A.link[pos] = make_uint2(sn.ci, rel | ((uint32_t)(g & 1) << 24) | ((sn.shared >> m & 1u) << 25) |
                                                ((uint32_t)sn.in_band << 26));
        }
        __syncthreads();
        if (threadIdx.x < LINK_GROUPS) run[threadIdx.x] += sh[threadIdx.x][32];
        __syncthreads();
    });
    // pad every group to its chunks
    for (int g = 0; g < LINK_GROUPS; ++g) {
        size_t gi = (size_t)p * LINK_GROUPS + g;
        uint32_t base = A.offset[gi], end = base + A.count[gi];
        for (uint32_t k = base + run[g] + threadIdx.x; k < end; k += blockDim.x) A.link[k] = make_uint2(NONE, 0u);
    }
    __syncthreads();
    // label the chunks with their direction (| 64 for a chunk of maybe
    // links, | 128 when a chunk holds an in_band link) and tag the sphere's
    // warps
    for (int g = 0; g < LINK_GROUPS; ++g) {
        size_t gi = (size_t)p * LINK_GROUPS + g;
        uint32_t base = A.offset[gi], end = base + A.count[gi];
        for (uint32_t k = base / 32 + wid; k < end / 32; k += nwarp) {
            uint32_t fl = __ballot_sync(0xffffffffu, ((A.link[32 * k + lane].y >> 26) & 1u) != 0u);
            if (lane == 0) A.chunk_dir[k] = (uint8_t)((g >> 1) | ((g & 1) ? 64 : 0) | (fl ? 128 : 0));
        }
    }
    uint32_t first = A.offset[(size_t)p * LINK_GROUPS];
    uint32_t last = A.offset[(size_t)p * LINK_GROUPS + LINK_GROUPS - 1] +
                    A.count[(size_t)p * LINK_GROUPS + LINK_GROUPS - 1];
    for (uint32_t k = first / LINK_WARP + threadIdx.x; k < last / LINK_WARP; k += blockDim.x) A.warp_p[k] = (uint32_t)p;
}

__global__ void k_fill_u64(unsigned long long* p, unsigned long long v, size_t n) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

void launch_paint(const PaintArgs& A, int n, size_t N, cudaStream_t s) {
    if (n <= 0) return;
    if (A.owner) k_fill_u64<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(A.best, ~0ull, N);
    k_paint<0><<<n, BOX_THREADS, 0, s>>>(A);
    if (A.owner) k_paint<1><<<n, BOX_THREADS, 0, s>>>(A);
}

void launch_words(const LayoutArgs& A, cudaStream_t s) {
    size_t W = (size_t)A.nx * A.ny * A.nw;
    k_words<<<(unsigned)((W + 255) / 256), 256, 0, s>>>(A);
}

void launch_words_bases(const LayoutArgs& A, uint32_t nA, cudaStream_t s) {
    size_t W = (size_t)A.nx * A.ny * A.nw;
    k_words_bases<<<(unsigned)((W + 255) / 256), 256, 0, s>>>(A, nA);
}

void launch_coords(const LayoutArgs& A, uint32_t nA, uint32_t nSpad, uint32_t* fbits, cudaStream_t s) {
    size_t W = (size_t)A.nx * A.ny * A.nw;
    k_coords<<<(unsigned)((W + 255) / 256), 256, 0, s>>>(A);
    uint32_t nwords = nSpad / 32;
    k_fbits<<<(nwords + 255) / 256, 256, 0, s>>>(fbits, nA, nwords);
}

void launch_gather_old(const Lat& Lnew, const Lat& Lold, cudaStream_t s) {
    if (!Lnew.nA) return;
    unsigned blocks = (Lnew.nA + 255) / 256;
    if (Lnew.st == 0)  // the populations move as stored (no conversion)
        k_gather_old<float><<<blocks, 256, 0, s>>>(Lnew, Lold);
    else
        k_gather_old<uint16_t><<<blocks, 256, 0, s>>>(Lnew, Lold);
}

void launch_band_collect(const LayoutArgs& A, uint32_t* band_coord, uint32_t* count, uint32_t cap,
                         cudaStream_t s) {
    size_t N = (size_t)A.nx * A.ny * A.nz;
    k_band_collect<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(A, band_coord, count, cap);
}

void launch_surf_count(const SurfArgs& A, int n, cudaStream_t s) {
    if (n > 0) k_surf_count<<<n, BOX_THREADS, 0, s>>>(A);
}

void launch_surf_fill(const SurfArgs& A, int n, cudaStream_t s) {
    if (n > 0) k_surf_fill<<<n, BOX_THREADS, 0, s>>>(A);
}

}  // namespace lbmdem
