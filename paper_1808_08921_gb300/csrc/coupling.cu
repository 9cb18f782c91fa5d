// coupling.cu -- fluid-solid coupling (Section 2.3).
//
//  * k_links: walks each sphere's link lists (one warp per 32 links of one
//    sphere in one direction).  For every fluid node x and direction d whose
//    neighbour x + c_d belongs to the sphere, slot opp(d) of x holds the
//    post-collision value f~_d(x) (AA layout, either parity); it is replaced
//    by the bounced value f~_d - 6 w_d rho_f c_d . V_b (Eq. 14, moving wall
//    with V_b = V + Omega x (x_b - X), x_b = x + c_d / 2), and the link force
//    c_d (f~_d + f_bounced - 2 w_d rho_f) (Eq. 15, counted about the rest
//    state: the mean pressure acts on the whole grain, and with populations
//    stored as deviations from w_d rho_f this is c_d (2 g~_d - delta)) and
//    its torque (Eq. 19) are summed by warp shuffles, then one FP64 atomic
//    per warp per component.
//  * map update: every node within `skin` of a sphere surface is re-tested
//    against the current sphere positions (where spheres overlap, the one
//    with the smallest |x - X|^2 / R^2 owns the node, the lowest index on a
//    tie; the inlet/outlet planes stay fluid).  Changed nodes are
//    queued; for each, the natural populations of the node and its 18
//    neighbours are gathered with the old map, the conversion is applied
//    (covered node: its momentum goes to the sphere, Eq. 16; uncovered node:
//    equilibrium at the mean density of its fluid neighbours and the surface
//    velocity, the sphere loses that momentum, Eq. 17), the map is committed,
//    and the populations are scattered back with the new map (in the AA
//    layout the slot of a population depends on whether its upstream
//    neighbour is fluid).
#include "common.cuh"
#include "kernels.cuh"

namespace lbmdem {

__device__ __forceinline__ int imin_wrap(int d, int L) {
    // minimum image of an integer offset (any magnitude)
    d %= L;
    if (d < 0) d += L;
    if (d > L / 2) d -= L;
    return d;
}

// Direction m at run time (warp-uniform in the link kernel), from bit masks of
// the velocity set of Eq. 3: one compact body instead of 18 specialisations
// keeps the kernel inside the instruction cache.
constexpr uint32_t DPX = (1u << 0) | (1u << 6) | (1u << 7) | (1u << 8) | (1u << 9);
constexpr uint32_t DNX = (1u << 1) | (1u << 10) | (1u << 11) | (1u << 12) | (1u << 13);
constexpr uint32_t DPY = (1u << 2) | (1u << 6) | (1u << 10) | (1u << 14) | (1u << 15);
constexpr uint32_t DNY = (1u << 3) | (1u << 7) | (1u << 11) | (1u << 16) | (1u << 17);
constexpr uint32_t DPZ = (1u << 4) | (1u << 8) | (1u << 12) | (1u << 14) | (1u << 16);
constexpr uint32_t DNZ = (1u << 5) | (1u << 9) | (1u << 13) | (1u << 15) | (1u << 17);
// opposites, 5 bits each: m 0..11 in the low word, 12..18 in the high word
constexpr unsigned long long DOLO = 1ull | (0ull << 5) | (3ull << 10) | (2ull << 15) | (5ull << 20) |
                                    (4ull << 25) | (11ull << 30) | (10ull << 35) | (13ull << 40) |
                                    (12ull << 45) | (7ull << 50) | (6ull << 55);
constexpr unsigned long long DOHI = 9ull | (8ull << 5) | (17ull << 10) | (16ull << 15) | (15ull << 20) |
                                    (14ull << 25) | (18ull << 30);
__host__ __device__ constexpr int rcx(int m) { return (int)((DPX >> m) & 1u) - (int)((DNX >> m) & 1u); }
__host__ __device__ constexpr int rcy(int m) { return (int)((DPY >> m) & 1u) - (int)((DNY >> m) & 1u); }
__host__ __device__ constexpr int rcz(int m) { return (int)((DPZ >> m) & 1u) - (int)((DNZ >> m) & 1u); }
__host__ __device__ constexpr int ropp(int m) {
    return m < 12 ? (int)((DOLO >> (5 * m)) & 31ull) : (int)((DOHI >> (5 * (m - 12))) & 31ull);
}
constexpr bool dir_tables_agree(int m) {
    return m == Q ? true
                  : (rcx(m) == cx(m) && rcy(m) == cy(m) && rcz(m) == cz(m) && ropp(m) == opp(m) &&
                     dir_tables_agree(m + 1));
}
static_assert(dir_tables_agree(0), "run-time direction decoding disagrees with Eq. 3 tables");

struct Dir {
    int cx, cy, cz, op;
    float w;
    __device__ __forceinline__ explicit Dir(int m) {
        cx = rcx(m);
        cy = rcy(m);
        cz = rcz(m);
        op = ropp(m);
        w = (cx * cx + cy * cy + cz * cz) == 1 ? 1.0f / 18.0f : 1.0f / 36.0f;
    }
};

// LINK_WARP / 32 links per thread, all of sphere p in direction d.  The
// phases (records, fluid bits, ownership, populations, updates) each issue
// all of the thread's loads before using any, so the K chains overlap.
__device__ __noinline__ void link_warp(const Lat& L, const PartView& P, const LinkLists& B, uint32_t w, int p,
                                       const Dir& d, float* acc) {
    constexpr int K = LINK_WARP / 32;
    const uint32_t lane = threadIdx.x & 31;
    const uint2* rec = B.link + (size_t)w * LINK_WARP + lane;
    uint2 lk[K];
#pragma unroll
    for (int k = 0; k < K; ++k) lk[k] = __ldcs(&rec[k * 32]);
    uint32_t fb[K];
#pragma unroll
    for (int k = 0; k < K; ++k) fb[k] = lk[k].x != NONE ? __ldg(&L.fbits[lk[k].x >> 5]) : 0u;
    float4 xf = P.xf[p];
    float4 V = P.V[p], W = P.W[p];
    const float R2 = __fmul_rn(P.R[p], P.R[p]);
    bool on[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        on[k] = lk[k].x != NONE && ((fb[k] >> (lk[k].x & 31)) & 1u);
        if (on[k] && (lk[k].y >> 24 & 1u)) {  // band neighbour: does the sphere own it now?
            int ix = (int)(lk[k].y & 255u) - 128, iy = (int)((lk[k].y >> 8) & 255u) - 128,
                iz = (int)((lk[k].y >> 16) & 255u) - 128;
            bool read_owner = (lk[k].y >> 25 & 1u) != 0;  // another sphere may claim it
            if (!read_owner) {
                // the map update's FP32 test, same operands and rounding
                float ax = __fsub_rn((float)(ix + d.cx), xf.x), ay = __fsub_rn((float)(iy + d.cy), xf.y),
                      az = __fsub_rn((float)(iz + d.cz), xf.z);
                float d2 = norm2_rn(ax, ay, az);
                if (fabsf(d2 - R2) <= FP32_MARGIN * R2)
                    read_owner = true;
                else
                    on[k] = d2 < R2;
            }
            if (read_owner) {
                int4 o = P.orgw[p];  // wrapped origin: the offsets are small
                int xs = o.x + ix + d.cx, ys = o.y + iy + d.cy, zs = o.z + iz + d.cz;
                if (L.px) xs = xs < 0 ? xs + L.nx : (xs >= L.nx ? xs - L.nx : xs);
                ys = ys < 0 ? ys + L.ny : (ys >= L.ny ? ys - L.ny : ys);
                zs = zs < 0 ? zs + L.nz : (zs >= L.nz ? zs - L.nz : zs);
                on[k] = L.owner[((size_t)xs * L.ny + ys) * L.nz + zs] == p;
            }
        }
    }
    float* plane = L.f + (size_t)d.op * L.nSpad;
    float v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = on[k] ? plane[lk[k].x] : 0.f;
    const float c6w = 6.0f * L.rho_f * d.w;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (!on[k]) continue;
        int ix = (int)(lk[k].y & 255u) - 128, iy = (int)((lk[k].y >> 8) & 255u) - 128,
            iz = (int)((lk[k].y >> 16) & 255u) - 128;
        float rx = (float)ix - xf.x, ry = (float)iy - xf.y, rz = (float)iz - xf.z;
        float bx = rx + 0.5f * d.cx, by = ry + 0.5f * d.cy, bz = rz + 0.5f * d.cz;
        float cv = d.cx * (V.x + (W.y * bz - W.z * by)) + d.cy * (V.y + (W.z * bx - W.x * bz)) +
                   d.cz * (V.z + (W.x * by - W.y * bx));
        float delta = c6w * cv;
        plane[lk[k].x] = v[k] - delta;
        float q = 2.0f * v[k] - delta;
        float qx = d.cx * q, qy = d.cy * q, qz = d.cz * q;
        acc[0] += qx;
        acc[1] += qy;
        acc[2] += qz;
        // b x (c q) = r x (c q) since c x c = 0
        acc[3] += ry * qz - rz * qy;
        acc[4] += rz * qx - rx * qz;
        acc[5] += rx * qy - ry * qx;
    }
}

// One warp: LINK_WARP links of one sphere in one direction (no divergence
// between lanes); warp-shuffle sums, then one FP64 atomic per component per
// warp into one of NREP accumulator copies of the sphere.
__global__ void __launch_bounds__(256) k_links(Lat L, PartView P, LinkLists B) {
    uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= B.nwarps) return;  // whole warps
    uint32_t pd = B.warp_pd[w];
    int p = (int)(pd >> 5);
    Dir d((int)(pd & 31u));
    float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    link_warp(L, P, B, w, p, d, acc);
    const unsigned full = 0xffffffffu;
#pragma unroll
    for (int o = 16; o; o >>= 1)
#pragma unroll
        for (int c = 0; c < 6; ++c) acc[c] += __shfl_xor_sync(full, acc[c], o);
    if ((threadIdx.x & 31) == 0) {
        size_t rep = (size_t)(w % NREP) * P.n + p;
        double* F = P.Fh + 3 * rep;
        double* T = P.Th + 3 * rep;
        atomicAdd(F + 0, (double)acc[0]);
        atomicAdd(F + 1, (double)acc[1]);
        atomicAdd(F + 2, (double)acc[2]);
        atomicAdd(T + 0, (double)acc[3]);
        atomicAdd(T + 1, (double)acc[4]);
        atomicAdd(T + 2, (double)acc[5]);
    }
}

void launch_links(const Lat& L, const PartView& P, const LinkLists& B, cudaStream_t s) {
    if (B.nwarps == 0) return;
    uint64_t threads = (uint64_t)B.nwarps * 32;  // one warp per LINK_WARP links
    k_links<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(L, P, B);
}

// ------------------------------------------------------------ map update

// Current centre of sphere p in FP64 and the node's offset to it along one
// axis, taken to the nearest periodic image and rounded once: (y + k L) - X.
__device__ __forceinline__ double node_offset(int y, double X, int Lax, int periodic) {
    if (!periodic) return (double)y - X;
    double k = floor((X - (double)y) / (double)Lax + 0.5);
    return (double)(y + (int)k * Lax) - X;
}

__device__ __forceinline__ void centre(const PartView& P, int p, double& X0, double& X1, double& X2) {
    float4 d = P.dX[p], c = P.dXc[p];
    X0 = P.Xref[3 * p] + (double)d.x - (double)c.x;
    X1 = P.Xref[3 * p + 1] + (double)d.y - (double)c.y;
    X2 = P.Xref[3 * p + 2] + (double)d.z - (double)c.z;
}

struct MapArgs {
    Lat L;
    PartView P;
    Band band;
    FlipBuf F;
    DevStats* st;
    int par;        // parity of the step (selects the flip counter)
    int after_even; // layout of the state the step starts from
};

__global__ void k_map_band(MapArgs A) {
    uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) A.st->nflip[A.par ^ 1] = 0;
    if (k < (uint32_t)A.P.n) {
        for (int r = 0; r < NREP; ++r)
            for (int a = 0; a < 3; ++a) {
                A.P.Fh[3 * ((size_t)r * A.P.n + k) + a] = 0.0;
                A.P.Th[3 * ((size_t)r * A.P.n + k) + a] = 0.0;
            }
    }
    if (k >= A.band.n) return;
    const Lat& L = A.L;
    int x, y, z;
    unpack_coord(A.band.coord[k], x, y, z);
    int4 cand = A.band.cand[k];
    int c4[4] = {cand.x, cand.y, cand.z, cand.w};
    int best = OWNER_FLUID;
    if (L.px || (x > 0 && x < L.nx - 1)) {
        // FP32 test in each sphere's lattice frame (node - floor(Xref) - xf);
        // it decides only where its margin (1e-5 of R^2, ~100x its rounding)
        // guarantees the FP64 answer, else the exact FP64 rule decides
        bool exact = false;
        float bestr = 0.f;
        for (int a = 0; a < 4; ++a) {
            int p = c4[a];
            if (p < 0) break;
            int4 o = A.P.org[p];
            float4 xf = A.P.xf[p];
            int ix = L.px ? imin_wrap(x - o.x, L.nx) : x - o.x;
            int iy = imin_wrap(y - o.y, L.ny), iz = imin_wrap(z - o.z, L.nz);
            float ax = __fsub_rn((float)ix, xf.x), ay = __fsub_rn((float)iy, xf.y), az = __fsub_rn((float)iz, xf.z);
            float d2 = norm2_rn(ax, ay, az);
            float R2 = __fmul_rn(A.P.R[p], A.P.R[p]);
            if (fabsf(d2 - R2) <= FP32_MARGIN * R2) {
                exact = true;
                break;
            }
            if (d2 < R2) {
                float r = d2 / R2;
                if (best != OWNER_FLUID && fabsf(r - bestr) <= 1e-5f) {
                    exact = true;
                    break;
                }
                if (best == OWNER_FLUID || r < bestr) {
                    best = p;
                    bestr = r;
                }
            }
        }
        if (exact) {
            best = OWNER_FLUID;
            double best_ratio = 0.0;
            for (int a = 0; a < 4; ++a) {  // candidates ascend: ties keep the lowest index
                int p = c4[a];
                if (p < 0) break;
                double X0, X1, X2;
                centre(A.P, p, X0, X1, X2);
                double ax = node_offset(x, X0, L.nx, L.px);
                double ay = node_offset(y, X1, L.ny, 1);
                double az = node_offset(z, X2, L.nz, 1);
                double Rp = A.P.Rd[p];
                if (inside_exact(ax, ay, az, Rp)) {
                    double r = inside_ratio(ax, ay, az, Rp);
                    if (best == OWNER_FLUID || r < best_ratio) {
                        best = p;
                        best_ratio = r;
                    }
                }
            }
        }
    }
    size_t li = ((size_t)x * L.ny + y) * L.nz + z;
    int old = L.owner[li];
    if (old != best) {
        uint32_t slot = atomicAdd(&A.st->nflip[A.par], 1u);
        if (slot < A.F.cap) {
            Flip f;
            f.coord = A.band.coord[k];
            f.old_owner = old;
            f.new_owner = best;
            f.pad = 0;
            A.F.rec[slot] = f;
        } else {
            atomicOr(&A.st->status, ST_CAPACITY);
        }
    }
}

// One warp per queued node: lanes 0..18 gather the node (lane 18, c = 0)
// and its 18 neighbours with the old map; lane 0 applies the conversion.
__device__ void map_gather_convert_one(const MapArgs& A, uint32_t w, int lane) {
    const Lat& L = A.L;
    Flip f = A.F.rec[w];
    int x, y, z;
    unpack_coord(f.coord, x, y, z);
    float* sc = A.F.scratch + (size_t)w * Q * Q;
    bool valid = false;
    float rho_j = 0.f;
    if (lane < Q) {
        int xs = x + cx(lane), ys = wrap1(y + cy(lane), L.ny), zs = wrap1(z + cz(lane), L.nz);
        bool in = true;
        if (L.px) xs = wrap1(xs, L.nx);
        else in = xs >= 0 && xs < L.nx;
        if (in) {
            bool fl;
            uint32_t ci = stored_index(L, xs, ys, zs, fl);
            if (fl && ci != NONE) {
                float s = 0.f;
#pragma unroll
                for (int m = 0; m < Q; ++m) {
                    float g = *pop_loc(L, A.after_even, xs, ys, zs, ci, m);
                    sc[lane * Q + m] = g;
                    s += g;
                }
                rho_j = L.rho_f + s;
                valid = true;
            }
        }
    }
    const unsigned full = 0xffffffffu;
    // mean density of the fluid neighbours (not the node itself)
    float rs = (lane < Q - 1 && valid) ? rho_j : 0.f;
    float rc = (lane < Q - 1 && valid) ? 1.f : 0.f;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        rs += __shfl_xor_sync(full, rs, o);
        rc += __shfl_xor_sync(full, rc, o);
    }
    __syncwarp();
    if (lane < Q) A.F.valid[(size_t)w * Q + lane] = valid ? 1 : 0;
    __syncwarp();  // lane 0 may set the node's own flag below
    if (lane != 0) return;
    int o = f.old_owner, nw = f.new_owner;
    if (o == OWNER_FLUID && nw != OWNER_FLUID) {
        // covered: the sphere gains the node's momentum (Eq. 16)
        const float* g = sc + 18 * Q;
        double j[3] = {0, 0, 0};
        for (int m = 0; m < Q; ++m) {
            j[0] += cx(m) * (double)g[m];
            j[1] += cy(m) * (double)g[m];
            j[2] += cz(m) * (double)g[m];
        }
        double X0, X1, X2;
        centre(A.P, nw, X0, X1, X2);
        double r[3] = {node_offset(x, X0, L.nx, L.px), node_offset(y, X1, L.ny, 1),
                       node_offset(z, X2, L.nz, 1)};
        atomicAdd(&A.P.Fh[3 * nw], j[0]);
        atomicAdd(&A.P.Fh[3 * nw + 1], j[1]);
        atomicAdd(&A.P.Fh[3 * nw + 2], j[2]);
        atomicAdd(&A.P.Th[3 * nw], r[1] * j[2] - r[2] * j[1]);
        atomicAdd(&A.P.Th[3 * nw + 1], r[2] * j[0] - r[0] * j[2]);
        atomicAdd(&A.P.Th[3 * nw + 2], r[0] * j[1] - r[1] * j[0]);
    } else if (o != OWNER_FLUID && nw == OWNER_FLUID) {
        // uncovered: equilibrium at rho_bar and the surface velocity (Eq. 17)
        double rb = rc > 0.f ? (double)rs / (double)rc : (double)L.rho_f;
        double X0, X1, X2;
        centre(A.P, o, X0, X1, X2);
        double r[3] = {node_offset(x, X0, L.nx, L.px), node_offset(y, X1, L.ny, 1),
                       node_offset(z, X2, L.nz, 1)};
        float4 V = A.P.V[o], W = A.P.W[o];
        double vb[3] = {V.x + (W.y * r[2] - W.z * r[1]), V.y + (W.z * r[0] - W.x * r[2]),
                        V.z + (W.x * r[1] - W.y * r[0])};
        float rbf = (float)rb;
        float ux = (float)vb[0], uy = (float)vb[1], uz = (float)vb[2];
        float uu15 = 1.5f * (ux * ux + uy * uy + uz * uz);
        float* g = sc + 18 * Q;
        for (int m = 0; m < Q; ++m) {
            float cu = cx(m) * ux + cy(m) * uy + cz(m) * uz;
            g[m] = wt(m) * ((rbf - L.rho_f) + rbf * (3.f * cu + 4.5f * cu * cu - uu15));
        }
        A.F.valid[(size_t)w * Q + 18] = 1;
        double mom[3] = {rb * vb[0], rb * vb[1], rb * vb[2]};
        atomicAdd(&A.P.Fh[3 * o], -mom[0]);
        atomicAdd(&A.P.Fh[3 * o + 1], -mom[1]);
        atomicAdd(&A.P.Fh[3 * o + 2], -mom[2]);
        atomicAdd(&A.P.Th[3 * o], -(r[1] * mom[2] - r[2] * mom[1]));
        atomicAdd(&A.P.Th[3 * o + 1], -(r[2] * mom[0] - r[0] * mom[2]));
        atomicAdd(&A.P.Th[3 * o + 2], -(r[0] * mom[1] - r[1] * mom[0]));
    }
}

__global__ void k_map_gather_convert(MapArgs A) {
    int lane = threadIdx.x & 31;
    uint32_t nf = min(A.st->nflip[A.par], A.F.cap);
    uint32_t nwarp = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nf; w += nwarp)
        map_gather_convert_one(A, w, lane);
}

__device__ void map_commit_one(const MapArgs& A, uint32_t k);

__global__ void k_map_commit(MapArgs A) {
    uint32_t nf = min(A.st->nflip[A.par], A.F.cap);
    uint32_t t0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (t0 == 0) atomicAdd(&A.st->flips_total, (unsigned long long)nf);
    for (uint32_t k = t0; k < nf; k += gridDim.x * blockDim.x) map_commit_one(A, k);
}

__device__ void map_commit_one(const MapArgs& A, uint32_t k) {
    const Lat& L = A.L;
    Flip f = A.F.rec[k];
    int x, y, z;
    unpack_coord(f.coord, x, y, z);
    size_t li = ((size_t)x * L.ny + y) * L.nz + z;
    bool fl;
    uint32_t ci = stored_index(L, x, y, z, fl);
    uint32_t wi = ((uint32_t)x * L.ny + y) * L.nw + (z >> 5);
    uint32_t bit = 1u << (z & 31);
    if (f.new_owner == OWNER_FLUID) {
        if (ci == NONE) {  // would need a node outside the stored set
            atomicOr(&A.st->status, ST_SKIN);
            return;
        }
        atomicOr(&L.rec[wi].x, bit);
        atomicOr(&L.fbits[ci >> 5], 1u << (ci & 31));
    } else if (f.old_owner == OWNER_FLUID) {
        atomicAnd(&L.rec[wi].x, ~bit);
        if (ci != NONE) atomicAnd(&L.fbits[ci >> 5], ~(1u << (ci & 31)));
    }
    L.owner[li] = f.new_owner;
}

__device__ void map_scatter_one(const MapArgs& A, uint32_t w, int lane);

__global__ void k_map_scatter(MapArgs A) {
    int lane = threadIdx.x & 31;
    uint32_t nf = min(A.st->nflip[A.par], A.F.cap);
    uint32_t nwarp = (gridDim.x * blockDim.x) >> 5;
    if (lane >= Q) return;
    for (uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nf; w += nwarp)
        map_scatter_one(A, w, lane);
}

__device__ void map_scatter_one(const MapArgs& A, uint32_t w, int lane) {
    if (!A.F.valid[(size_t)w * Q + lane]) return;
    const Lat& L = A.L;
    Flip f = A.F.rec[w];
    int x, y, z;
    unpack_coord(f.coord, x, y, z);
    int xs = x + cx(lane), ys = wrap1(y + cy(lane), L.ny), zs = wrap1(z + cz(lane), L.nz);
    if (L.px) xs = wrap1(xs, L.nx);
    bool fl;
    uint32_t ci = stored_index(L, xs, ys, zs, fl);
    if (!fl || ci == NONE) return;
    const float* sc = A.F.scratch + (size_t)w * Q * Q + lane * Q;
#pragma unroll
    for (int m = 0; m < Q; ++m) *pop_loc(L, A.after_even, xs, ys, zs, ci, m) = sc[m];
}

void launch_map_update(const Lat& L, const PartView& P, const Band& band, const FlipBuf& F,
                       DevStats* st, bool after_even, int step_parity, cudaStream_t s) {
    MapArgs A{L, P, band, F, st, step_parity, after_even ? 1 : 0};
    uint32_t nb = band.n > (uint32_t)P.n ? band.n : (uint32_t)P.n;
    if (nb == 0) nb = 1;
    k_map_band<<<(nb + 255) / 256, 256, 0, s>>>(A);
    if (band.n == 0) return;
    // the queued count is read on the device: fixed grids stride over it
    const unsigned grid = 2 * 152;
    k_map_gather_convert<<<grid, 256, 0, s>>>(A);
    k_map_commit<<<grid, 256, 0, s>>>(A);
    k_map_scatter<<<grid, 256, 0, s>>>(A);
}

}  // namespace lbmdem
