// coupling.cu -- fluid-solid coupling (Section 2.3).
//
//  * k_links: walks each sphere's link lists (one warp per LINK_WARP links of
//    one sphere, in chunks of 32 links of one direction).  For every fluid
//    node x and direction d whose neighbour x + c_d belongs to the sphere,
//    slot opp(d) of x holds the post-collision value f~_d(x) (AA layout,
//    either parity); it is replaced
//    by the bounced value f~_d - 6 w_d rho_f c_d . V_b (Eq. 14, moving wall
//    with V_b = V + Omega x (x_b - X), x_b = x + c_d / 2), and the link force
//    c_d (f~_d + f_bounced - 2 w_d rho_f) (Eq. 15, counted about the rest
//    state: the mean pressure acts on the whole grain, and with populations
//    stored as deviations from w_d rho_f this is c_d (2 g~_d - delta)) and
//    its torque (Eq. 19) are summed by warp shuffles, then one FP64 atomic
//    per warp per component.
//  * map update: the nodes within `skin` of a sphere surface (the band) are
//    re-tested against the current sphere positions -- after a layout all of
//    them, later only those no farther from a candidate surface than the
//    largest displacement since the layout -- (where spheres overlap, the one
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



// Directions of Eq. 3 as a constant table, read with a warp-uniform index.
struct DirC {
    float cx, cy, cz, w;
    int op;
};
__constant__ DirC kDir[Q - 1] = {
#define LBMDEM_DIR(m) {(float)cx(m), (float)cy(m), (float)cz(m), wt(m), opp(m)}
    LBMDEM_DIR(0),  LBMDEM_DIR(1),  LBMDEM_DIR(2),  LBMDEM_DIR(3),  LBMDEM_DIR(4),  LBMDEM_DIR(5),
    LBMDEM_DIR(6),  LBMDEM_DIR(7),  LBMDEM_DIR(8),  LBMDEM_DIR(9),  LBMDEM_DIR(10), LBMDEM_DIR(11),
    LBMDEM_DIR(12), LBMDEM_DIR(13), LBMDEM_DIR(14), LBMDEM_DIR(15), LBMDEM_DIR(16), LBMDEM_DIR(17),
#undef LBMDEM_DIR
};

// the same directions as 16-byte global entries {cx, cy, cz, opposite}: one
// 128-bit load per chunk in the link kernel's main loop
__device__ const float4 kDirV[Q - 1] = {
#define LBMDEM_DIRV(m) {(float)cx(m), (float)cy(m), (float)cz(m), (float)opp(m)}
    LBMDEM_DIRV(0),  LBMDEM_DIRV(1),  LBMDEM_DIRV(2),  LBMDEM_DIRV(3),  LBMDEM_DIRV(4),  LBMDEM_DIRV(5),
    LBMDEM_DIRV(6),  LBMDEM_DIRV(7),  LBMDEM_DIRV(8),  LBMDEM_DIRV(9),  LBMDEM_DIRV(10), LBMDEM_DIRV(11),
    LBMDEM_DIRV(12), LBMDEM_DIRV(13), LBMDEM_DIRV(14), LBMDEM_DIRV(15), LBMDEM_DIRV(16), LBMDEM_DIRV(17),
#undef LBMDEM_DIRV
};

// the LINK_CHUNKS direction bytes of warp w, in one load
__device__ __forceinline__ unsigned long long warp_chunk_dirs(const LinkLists& B, uint32_t w) {
    if (LINK_CHUNKS == 8) return *reinterpret_cast<const unsigned long long*>(B.chunk_dir + (size_t)w * 8);
    return *reinterpret_cast<const uint32_t*>(B.chunk_dir + (size_t)w * 4);
}

// b - 128 for the byte b at bit `shift` of a record word, exactly, as FP32
// (2^23 + b from the bits, minus 2^23 + 128: no conversion instruction).
__device__ __forceinline__ float rel_f(uint32_t word, int shift) {
    return __uint_as_float(0x4B000000u | ((word >> shift) & 255u)) - 8388736.0f;
}

// Does sphere p own the band neighbour x + c of the link node now (c the
// link's direction)?  Decided by the map update's FP32 test (same operands
// and rounding) away from its margin, else (or when several spheres may
// claim the node) by the owner map.
__device__ __forceinline__ bool owns_neighbour(const Lat& L, const PartView& P, int p, uint32_t y, const DirC& d,
                                               const float4& xf, float R2) {
    if (!(y >> 25 & 1u)) {
        float ax = __fsub_rn(rel_f(y, 0) + d.cx, xf.x), ay = __fsub_rn(rel_f(y, 8) + d.cy, xf.y),
              az = __fsub_rn(rel_f(y, 16) + d.cz, xf.z);
        float d2 = norm2_rn(ax, ay, az);
        if (fabsf(d2 - R2) > FP32_MARGIN * R2) return d2 < R2;
    }
    int ix = (int)(y & 255u) - 128, iy = (int)((y >> 8) & 255u) - 128, iz = (int)((y >> 16) & 255u) - 128;
    int4 o = P.orgw[p];  // wrapped origin: the offsets are small
    int xs = o.x + ix + (int)d.cx, ys = o.y + iy + (int)d.cy, zs = o.z + iz + (int)d.cz;
    if (L.px) xs = xs < 0 ? xs + L.nx : (xs >= L.nx ? xs - L.nx : xs);
    ys = ys < 0 ? ys + L.ny : (ys >= L.ny ? ys - L.ny : ys);
    zs = zs < 0 ? zs + L.nz : (zs >= L.nz ? zs - L.nz : zs);
    return L.owner[((size_t)xs * L.ny + ys) * L.nz + zs] == p;
}

// One warp: LINK_WARP links of one sphere in chunks of 32, each chunk in one
// direction.  The phases (records, fluid bits, ownership, populations,
// updates) each issue all of the thread's loads before using any.  The
// moving-wall term of Eq. 14 at the link node x = origin + rel is
// 6 w rho_f c.(V + W x (b - X)) = alpha' + rel.beta, b = x + c/2 (c.(W x c)
// = 0), with alpha' and beta per (sphere, direction) from the map update.
// The torque (Eq. 19) is summed about the sphere's lattice origin and moved
// to the centre once per warp: sum r x (c q) = sum rel x (c q) - xf x F.
// Warp-shuffle sums, then one FP64 atomic per component per warp into one
// of NREP accumulator copies of the sphere.
// 56 registers (no spills): 36 resident warps per SM, more scattered
// loads in flight than the 32 warps at 64 registers (143.5 against 147 us
// on the 128 x 128 x 1024 column).
template <int ST>
__global__ void __maxnreg__(56) k_links(Lat L, PartView P, LinkLists B) {
    pdl_wait();
    pdl_trigger();
    constexpr int K = LINK_CHUNKS;
    auto* f = pops<ST>(L);
    // warps in reverse order: the last spheres' nodes were collided last and
    // are the likeliest to be still in L2
    const uint32_t w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w0 >= B.nwarps) return;  // whole warps
    const uint32_t w = B.nwarps - 1 - w0;
    const uint32_t lane = threadIdx.x & 31;
    const int p = (int)B.warp_p[w];
    const unsigned long long dirs = warp_chunk_dirs(B, w);
    const uint2* rec = B.link + (size_t)w * LINK_WARP + lane;
    uint2 lk[K];
#pragma unroll
    for (int k = 0; k < K; ++k) lk[k] = __ldcs(&rec[k * 32]);
    const float4 xf = P.xf[p];
    const float4* ab = P.ab + (size_t)p * (Q - 1);
    bool on[K];
#pragma unroll
    for (int k = 0; k < K; ++k) on[k] = lk[k].x != NONE;
    // the populations are loaded before the link is confirmed: a covered
    // link node keeps its slots, so the load is in bounds, and its latency
    // overlaps the fluid-bit and ownership checks
    float v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int op = (int)__ldg(&kDirV[(dirs >> (8 * k)) & 31u]).w;
        v[k] = on[k] ? to_f<ST>(f[(uint32_t)op * L.nSpad + lk[k].x], L.fsi) : 0.f;
    }
    if (dirs & 0xC0C0C0C0C0C0C0C0ull) {  // some chunk needs the fluid-bit or the ownership check
        uint32_t fb[K];
#pragma unroll
        for (int k = 0; k < K; ++k)  // only a node inside a band can have been covered
            fb[k] = on[k] && (lk[k].y >> 26 & 1u) ? __ldg(&L.fbits[lk[k].x >> 5]) : ~0u;
        const float R2 = __fmul_rn(P.R[p], P.R[p]);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            on[k] = on[k] && ((fb[k] >> (lk[k].x & 31)) & 1u);
            // a chunk of `maybe` links (whole chunks, so the branch is uniform)
            if ((dirs >> (8 * k)) & 64u)
                if (on[k]) on[k] = owns_neighbour(L, P, p, lk[k].y, kDir[(dirs >> (8 * k)) & 31u], xf, R2);
        }
    }
    float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const uint32_t m = (dirs >> (8 * k)) & 31u;
        const float4 dv = __ldg(&kDirV[m]);
        const DirC d = {dv.x, dv.y, dv.z, 0.f, (int)dv.w};
        const float4 a = ab[m];
        if (!on[k]) continue;
        const uint32_t y = lk[k].y;
        const float rx = rel_f(y, 0), ry = rel_f(y, 8), rz = rel_f(y, 16);
        const float delta = a.x + (rx * a.y + ry * a.z + rz * a.w);
        f[(uint32_t)d.op * L.nSpad + lk[k].x] = from_f<ST>(v[k] - delta, L.fs);
        const float q = 2.0f * v[k] - delta;
        const float qx = d.cx * q, qy = d.cy * q, qz = d.cz * q;
        acc[0] += qx;
        acc[1] += qy;
        acc[2] += qz;
        // b x (c q) = r x (c q) since c x c = 0; r = rel - xf
        acc[3] += ry * qz - rz * qy;
        acc[4] += rz * qx - rx * qz;
        acc[5] += rx * qy - ry * qx;
    }
    // torque about the centre, per lane (the correction is linear)
    acc[3] -= xf.y * acc[2] - xf.z * acc[1];
    acc[4] -= xf.z * acc[0] - xf.x * acc[2];
    acc[5] -= xf.x * acc[1] - xf.y * acc[0];
    // transposing butterfly: at each of the first three levels a lane keeps
    // half of its components and sends the other half, so the six sums (two
    // zero pads) take 4 + 2 + 1 + 1 + 1 shuffles; lane l ends with the warp
    // sum of component 4 b4 + 2 b3 + b2 (b = bits of l)
    const unsigned full = 0xffffffffu;
    float s8[8] = {acc[0], acc[1], acc[2], acc[3], acc[4], acc[5], 0.f, 0.f};
    {
        const bool up = lane & 16;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float keep = up ? s8[c + 4] : s8[c], send = up ? s8[c] : s8[c + 4];
            s8[c] = keep + __shfl_xor_sync(full, send, 16);
        }
    }
    {
        const bool up = lane & 8;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const float keep = up ? s8[c + 2] : s8[c], send = up ? s8[c] : s8[c + 2];
            s8[c] = keep + __shfl_xor_sync(full, send, 8);
        }
    }
    {
        const bool up = lane & 4;
        const float keep = up ? s8[1] : s8[0], send = up ? s8[0] : s8[1];
        s8[0] = keep + __shfl_xor_sync(full, send, 4);
    }
    s8[0] += __shfl_xor_sync(full, s8[0], 2);
    s8[0] += __shfl_xor_sync(full, s8[0], 1);
    const int comp = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
    if ((lane & 3) == 0 && comp < 6) {
        const size_t rep = (size_t)(w % NREP) * P.n + p;
        double* dst = comp < 3 ? P.Fh + 3 * rep + comp : P.Th + 3 * rep + (comp - 3);
        atomicAdd(dst, (double)s8[0]);
    }
}

void launch_links(const Lat& L, const PartView& P, const LinkLists& B, cudaStream_t s) {
    if (B.nwarps == 0) return;
    uint64_t threads = (uint64_t)B.nwarps * 32;  // one warp per LINK_WARP links
    // two-warp blocks: the warps' run times vary with their links' scatter,
    // and small blocks let the SMs refill as each pair finishes
    unsigned blocks = (unsigned)((threads + 63) / 64);
    if (L.st == 0) launch_pdl(k_links<0>, blocks, 64, s, L, P, B);
    else if (L.st == 1) launch_pdl(k_links<1>, blocks, 64, s, L, P, B);
    else launch_pdl(k_links<2>, blocks, 64, s, L, P, B);
}

// ------------------------------------------------------------ map update

// Current centre of sphere p in FP64 and the node's offset to it along one
// axis, taken to the nearest periodic image and rounded once: (y + k L) - X.
// The image count k is taken in FP32 (no FP64 division): it can differ from
// the exact one only for a node about half a box from the centre, which is
// outside every sphere and band (R + skin < L / 2), either image.
__device__ __forceinline__ double node_offset(int y, double X, int Lax, int periodic) {
    if (!periodic) return (double)y - X;
    float k = floorf((float)(X - (double)y) / (float)Lax + 0.5f);
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
    uint2* lw;      // link words renewed around converted nodes (null: not kept)
};

// Link word of the stored node (x, y, z) from the owner map (see LW_MASK):
// every direction whose neighbour a sphere owns is a link (out-of-range x
// neighbours of a non-periodic column are not).
__device__ uint2 link_word(const Lat& L, int x, int y, int z) {
    // every neighbour's owner is loaded before any is used
    int own[Q - 1];
#pragma unroll
    for (int m = 0; m < Q - 1; ++m) {
        int xs = x + cx(m);
        bool in = true;
        if (L.px) xs = wrap1(xs, L.nx);
        else in = xs >= 0 && xs < L.nx;
        const int ys = wrap1(y + cy(m), L.ny), zs = wrap1(z + cz(m), L.nz);
        own[m] = in ? __ldcg(&L.owner[((size_t)xs * L.ny + ys) * L.nz + zs]) : OWNER_FLUID;
    }
    uint32_t mask = 0u, sel = 0u, pa = LW_NONE, pb = LW_NONE;
    bool many = false;
#pragma unroll
    for (int m = 0; m < Q - 1; ++m) {
        if (own[m] == OWNER_FLUID) continue;
        mask |= 1u << m;
        const uint32_t p = (uint32_t)own[m];
        if (pa == LW_NONE || p == pa) {
            pa = p;
        } else if (pb == LW_NONE || p == pb) {
            pb = p;
            sel |= 1u << m;
        } else {
            many = true;
        }
    }
    if (many) {
        pa = LW_NONE;
        pb = LW_NONE;
        sel = 0u;
    }
    return make_uint2(mask | (pa << 18), sel | (pb << 18));
}

__global__ void k_link_words(Lat L, uint2* lw) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L.nS) return;
    int x, y, z;
    unpack_coord(L.coord[i], x, y, z);
    lw[i] = link_word(L, x, y, z);
}

void launch_link_words(const Lat& L, uint2* lw, cudaStream_t s) {
    if (L.nS) k_link_words<<<(L.nS + 255) / 256, 256, 0, s>>>(L, lw);
}

__global__ void k_map_band(MapArgs A) {
    pdl_trigger();  // launched normally: its predecessors are the DEM and the boundary branch
    uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) {
        A.st->nflip[A.par ^ 1] = 0;
        A.st->t += 1ull;  // the step starts: t counts it from here on
    }
    if (k < (uint32_t)A.P.n) {
        for (int r = 0; r < NREP; ++r)
            for (int a = 0; a < 3; ++a) {
                A.P.Fh[3 * ((size_t)r * A.P.n + k) + a] = 0.0;
                A.P.Th[3 * ((size_t)r * A.P.n + k) + a] = 0.0;
            }
        // moving-wall terms of this step's links of sphere k, per direction
        // m: beta = 6 w rho_f (c x W) and alpha' = 6 w rho_f c.V - xf.beta,
        // so that the term of Eq. 14 at a link node with offset rel from the
        // sphere's lattice origin is alpha' + rel.beta
        const float4 V = A.P.V[k], W = A.P.W[k], xf = A.P.xf[k];
        const float s6 = 6.0f * A.L.rho_f;
#pragma unroll
        for (int m = 0; m < Q - 1; ++m) {
            const float sw = s6 * wt(m);
            const float ex = (float)cx(m), ey = (float)cy(m), ez = (float)cz(m);
            const float bx = sw * (ey * W.z - ez * W.y), by = sw * (ez * W.x - ex * W.z),
                        bz = sw * (ex * W.y - ey * W.x);
            const float alpha = sw * (ex * V.x + ey * V.y + ez * V.z);
            A.P.ab[(size_t)k * (Q - 1) + m] = make_float4(alpha - (xf.x * bx + xf.y * by + xf.z * bz), bx, by, bz);
        }
        // the same state for the even steps' links inside the collide kernel
        const int4 o = A.P.orgw[k];
        A.P.pk[3 * (size_t)k] = make_float4(xf.x, xf.y, xf.z, V.x);
        A.P.pk[3 * (size_t)k + 1] = make_float4(V.y, V.z, W.x, W.y);
        A.P.pk[3 * (size_t)k + 2] = make_float4(W.z, __int_as_float(o.x), __int_as_float(o.y), __int_as_float(o.z));
    }
    if (k >= A.band.n) return;
    // a node farther from every candidate surface (at the layout) than any
    // sphere has moved since keeps its owner
    if (!A.st->layout_fresh) {
        const float moved = __uint_as_float(A.st->disp_layout_bits);
        if (A.band.slack[k] > moved + 1e-5f * (1.f + moved)) return;
    }
    const Lat& L = A.L;
    int x, y, z;
    unpack_coord(A.band.coord[k], x, y, z);
    const size_t li = ((size_t)x * L.ny + y) * L.nz + z;
    const int old = L.owner[li];  // issued early: independent of the test
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
            int4 o = A.P.orgw[p];  // origin wrapped into the box: |node - o| < L
            float4 xf = A.P.xf[p];
            int ix = L.px ? imin_small(x - o.x, L.nx) : x - o.x;
            int iy = imin_small(y - o.y, L.ny), iz = imin_small(z - o.z, L.nz);
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

// One block per queued node (grid-stride over the queue): thread t < 361
// gathers population m = t % 19 of node j = t / 19 with the old map, where
// j < 18 is the neighbour x + c_j and j = 18 the node itself; thread 361,
// idle during the gather, loads the sphere's state and the node's offset
// from its centre meanwhile and then applies the conversion.
constexpr int MAP_THREADS = 384;  // >= 19 * 19
template <int ST>
__global__ void __launch_bounds__(MAP_THREADS) k_map_gather_convert(MapArgs A) {
    pdl_wait();
    pdl_trigger();
    const Lat& L = A.L;
    __shared__ float sg[Q * Q];
    __shared__ float srho[Q];
    __shared__ int sv[Q];
    const uint32_t nf = min(A.st->nflip[A.par], A.F.cap);
    const int t = threadIdx.x, j = t / Q, m = t % Q;
    constexpr int CT = Q * Q;  // the converting thread
    for (uint32_t w = blockIdx.x; w < nf; w += gridDim.x) {
        const Flip f = A.F.rec[w];
        int x, y, z;
        unpack_coord(f.coord, x, y, z);
        float* sc = A.F.scratch + (size_t)w * Q * Q;
        const int o = f.old_owner, nw = f.new_owner;
        const int ps = o != OWNER_FLUID ? o : nw;  // the sphere that gains or loses the node
        double r[3] = {0.0, 0.0, 0.0};
        float4 V = make_float4(0.f, 0.f, 0.f, 0.f), W = V;
        if (t == CT && ps != OWNER_FLUID) {
            double X0, X1, X2;
            centre(A.P, ps, X0, X1, X2);
            r[0] = node_offset(x, X0, L.nx, L.px);
            r[1] = node_offset(y, X1, L.ny, 1);
            r[2] = node_offset(z, X2, L.nz, 1);
            V = A.P.V[ps];
            W = A.P.W[ps];
        }
        if (t < Q * Q) {
            bool valid = false;
            float g = 0.f;
            int xs = x + cx(j), ys = wrap1(y + cy(j), L.ny), zs = wrap1(z + cz(j), L.nz);
            bool in = true;
            if (L.px) xs = wrap1(xs, L.nx);
            else in = xs >= 0 && xs < L.nx;
            if (in) {
                bool fl;
                uint32_t ci = stored_index(L, xs, ys, zs, fl);
                if (fl && ci != NONE) {
                    g = to_f<ST>(*pop_loc<ST>(L, A.after_even, xs, ys, zs, ci, m), L.fsi);
                    valid = true;
                }
            }
            sg[t] = g;
            if (valid) sc[t] = g;
            if (m == 0) sv[j] = valid ? 1 : 0;
        }
        __syncthreads();
        if (t < Q) {  // density of each gathered node
            float d = 0.f;
            for (int mm = 0; mm < Q; ++mm) d += sg[t * Q + mm];
            srho[t] = L.rho_f + d;
        }
        __syncthreads();
        if (t == CT) {
            // mean density of the fluid neighbours (not the node itself)
            float rs = 0.f, rc = 0.f;
            for (int jj = 0; jj < Q - 1; ++jj) {
                if (!sv[jj]) continue;
                rs += srho[jj];
                rc += 1.f;
            }
            if (o == OWNER_FLUID && nw != OWNER_FLUID) {
                // covered: the sphere gains the node's momentum (Eq. 16)
                const float* g = sg + 18 * Q;
                float j0 = 0.f, j1 = 0.f, j2 = 0.f;
#pragma unroll
                for (int mm = 0; mm < Q; ++mm) {
                    j0 += cx(mm) * g[mm];
                    j1 += cy(mm) * g[mm];
                    j2 += cz(mm) * g[mm];
                }
                const double jm[3] = {j0, j1, j2};
                atomicAdd(&A.P.Fh[3 * nw], jm[0]);
                atomicAdd(&A.P.Fh[3 * nw + 1], jm[1]);
                atomicAdd(&A.P.Fh[3 * nw + 2], jm[2]);
                atomicAdd(&A.P.Th[3 * nw], r[1] * jm[2] - r[2] * jm[1]);
                atomicAdd(&A.P.Th[3 * nw + 1], r[2] * jm[0] - r[0] * jm[2]);
                atomicAdd(&A.P.Th[3 * nw + 2], r[0] * jm[1] - r[1] * jm[0]);
            } else if (o != OWNER_FLUID && nw == OWNER_FLUID) {
                // uncovered: equilibrium at rho_bar and the surface velocity (Eq. 17)
                const float rbf = rc > 0.f ? rs / rc : L.rho_f;
                const double rb = rbf;
                const float r0 = (float)r[0], r1 = (float)r[1], r2 = (float)r[2];
                const float ux = V.x + (W.y * r2 - W.z * r1), uy = V.y + (W.z * r0 - W.x * r2),
                            uz = V.z + (W.x * r1 - W.y * r0);
                const double vb[3] = {ux, uy, uz};
                float uu15 = 1.5f * (ux * ux + uy * uy + uz * uz);
                float* g = sc + 18 * Q;
                for (int mm = 0; mm < Q; ++mm) {
                    float cu = cx(mm) * ux + cy(mm) * uy + cz(mm) * uz;
                    g[mm] = wt(mm) * ((rbf - L.rho_f) + rbf * (3.f * cu + 4.5f * cu * cu - uu15));
                }
                sv[18] = 1;
                double mom[3] = {rb * vb[0], rb * vb[1], rb * vb[2]};
                atomicAdd(&A.P.Fh[3 * o], -mom[0]);
                atomicAdd(&A.P.Fh[3 * o + 1], -mom[1]);
                atomicAdd(&A.P.Fh[3 * o + 2], -mom[2]);
                atomicAdd(&A.P.Th[3 * o], -(r[1] * mom[2] - r[2] * mom[1]));
                atomicAdd(&A.P.Th[3 * o + 1], -(r[2] * mom[0] - r[0] * mom[2]));
                atomicAdd(&A.P.Th[3 * o + 2], -(r[0] * mom[1] - r[1] * mom[0]));
            }
        }
        __syncthreads();
        if (t < Q) A.F.valid[(size_t)w * Q + t] = (uint8_t)sv[t];
        __syncthreads();  // shared arrays are reused by the next queued node
    }
}

__device__ void map_commit_one(const MapArgs& A, uint32_t k);

__global__ void k_map_commit(MapArgs A) {
    pdl_wait();
    pdl_trigger();
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

// One block per queued node: thread t < 361 writes population m = t % 19 of
// node j = t / 19 back with the new map; the 19 first threads of the warp
// after those (a warp of its own, so neither path waits for the other)
// renew the link words of the node and its 18 neighbours from the committed
// owner map (neighbours shared by two queued nodes get the same word twice).
constexpr int SCATTER_THREADS = MAP_THREADS + 32;
template <int ST>
__global__ void __launch_bounds__(SCATTER_THREADS) k_map_scatter(MapArgs A) {
    pdl_wait();
    pdl_trigger();
    const Lat L = A.L;
    const uint32_t nf = min(A.st->nflip[A.par], A.F.cap);
    const int t = threadIdx.x, j = t / Q, m = t % Q;
    if (t >= Q * Q) {
        const int jn = t - MAP_THREADS;  // 0 ... 17: neighbour x + c_jn, 18: the node
        if (jn < 0) return;
        if (A.lw == nullptr || jn >= Q) return;
        for (uint32_t w = blockIdx.x; w < nf; w += gridDim.x) {
            int x, y, z;
            unpack_coord(A.F.rec[w].coord, x, y, z);
            int xs = x + cx(jn);
            if (L.px) xs = wrap1(xs, L.nx);
            else if (xs < 0 || xs >= L.nx) continue;
            const int ys = wrap1(y + cy(jn), L.ny), zs = wrap1(z + cz(jn), L.nz);
            bool fl;
            const uint32_t ci = stored_index(L, xs, ys, zs, fl);
            if (ci != NONE) A.lw[ci] = link_word(L, xs, ys, zs);
        }
        return;
    }
    for (uint32_t w = blockIdx.x; w < nf; w += gridDim.x) {
        if (!A.F.valid[(size_t)w * Q + j]) continue;
        const Flip f = A.F.rec[w];
        int x, y, z;
        unpack_coord(f.coord, x, y, z);
        int xs = x + cx(j), ys = wrap1(y + cy(j), L.ny), zs = wrap1(z + cz(j), L.nz);
        if (L.px) xs = wrap1(xs, L.nx);
        bool fl;
        uint32_t ci = stored_index(L, xs, ys, zs, fl);
        if (!fl || ci == NONE) continue;
        *pop_loc<ST>(L, A.after_even, xs, ys, zs, ci, m) = from_f<ST>(A.F.scratch[(size_t)w * Q * Q + t], L.fs);
    }
}

// Launch shapes: a column alone on the GPU takes small band blocks (most band
// nodes leave at the slack test, and small blocks keep the SMs busy with the
// few that go on to the sphere tests) and conversion grids of 4 x 152 blocks
// (a settling packing converts a few hundred nodes per step); columns of a
// batch, which share the GPU with each other, take 256-thread band blocks
// and 152 conversion blocks, fewer blocks to schedule beside the other
// columns' kernels.
void launch_map_update(const Lat& L, const PartView& P, const Band& band, const FlipBuf& F,
                       DevStats* st, bool after_even, int step_parity, uint2* lw, bool shared_gpu, cudaStream_t s) {
    MapArgs A{L, P, band, F, st, step_parity, after_even ? 1 : 0, lw};
    uint32_t nb = band.n > (uint32_t)P.n ? band.n : (uint32_t)P.n;
    if (nb == 0) nb = 1;
    const unsigned bb = shared_gpu ? 256 : 64;
    k_map_band<<<(nb + bb - 1) / bb, bb, 0, s>>>(A);
    if (band.n == 0) return;
    // the queued count is read on the device: fixed grids stride over it
    const unsigned grid = shared_gpu ? 152 : 4 * 152;
    if (L.st == 0) launch_pdl(k_map_gather_convert<0>, grid, MAP_THREADS, s, A);
    else if (L.st == 1) launch_pdl(k_map_gather_convert<1>, grid, MAP_THREADS, s, A);
    else launch_pdl(k_map_gather_convert<2>, grid, MAP_THREADS, s, A);
    launch_pdl(k_map_commit, grid, 256, s, A);
    const unsigned sthreads = lw ? SCATTER_THREADS : MAP_THREADS;
    if (L.st == 0) launch_pdl(k_map_scatter<0>, grid, sthreads, s, A);
    else if (L.st == 1) launch_pdl(k_map_scatter<1>, grid, sthreads, s, A);
    else launch_pdl(k_map_scatter<2>, grid, sthreads, s, A);
}

}  // namespace lbmdem
