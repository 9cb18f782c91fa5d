// coupling.cu -- fluid-solid coupling (Section 2.3).
//
//  * k_links: walks each sphere's list of surface nodes (one warp per 32
//    entries of one sphere).  For every fluid node x and direction d whose
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

__global__ void __launch_bounds__(256) k_links(Lat L, PartView P, LinkLists B) {
    uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t w = e >> 5;
    if (w >= B.nwarps) return;  // whole warps only
    int p = B.warp_part[w];
    uint2 ent = B.ent[e];
    float Fx = 0.f, Fy = 0.f, Fz = 0.f, Tx = 0.f, Ty = 0.f, Tz = 0.f;
    float4 xf = P.xf[p];
    if (ent.x != NONE && fluid_bit(L, ent.x)) {
        int x, y, z;
        unpack_coord(ent.y, x, y, z);
        int4 o = P.org[p];
        float4 V = P.V[p], W = P.W[p];
        float R = P.R[p];
        float Rm2 = (R + 0.01f) * (R + 0.01f);
        int ix = L.px ? imin_wrap(x - o.x, L.nx) : x - o.x;
        int iy = imin_wrap(y - o.y, L.ny), iz = imin_wrap(z - o.z, L.nz);
        float rx = (float)ix - xf.x, ry = (float)iy - xf.y, rz = (float)iz - xf.z;
        const float sixrho = 6.0f * L.rho_f;
#pragma unroll
        for (int m = 0; m < Q - 1; ++m) {
            float ax = rx + (float)cx(m), ay = ry + (float)cy(m), az = rz + (float)cz(m);
            if (ax * ax + ay * ay + az * az >= Rm2) continue;
            int xs = x + cx(m);
            if (L.px) xs = wrap1(xs, L.nx);
            else if (xs < 0 || xs >= L.nx) continue;
            int ys = wrap1(y + cy(m), L.ny), zs = wrap1(z + cz(m), L.nz);
            if (L.owner[((size_t)xs * L.ny + ys) * L.nz + zs] != p) continue;
            float* slot = L.f + (size_t)opp(m) * L.nSpad + ent.x;
            float v = *slot;
            float bx = rx + 0.5f * cx(m), by = ry + 0.5f * cy(m), bz = rz + 0.5f * cz(m);
            float vbx = V.x + (W.y * bz - W.z * by);
            float vby = V.y + (W.z * bx - W.x * bz);
            float vbz = V.z + (W.x * by - W.y * bx);
            float cv = (float)cx(m) * vbx + (float)cy(m) * vby + (float)cz(m) * vbz;
            float delta = wt(m) * sixrho * cv;
            *slot = v - delta;
            float q = 2.0f * v - delta;
            float qx = cx(m) * q, qy = cy(m) * q, qz = cz(m) * q;
            Fx += qx;
            Fy += qy;
            Fz += qz;
            // b x (c q) = r x (c q) since c x c = 0
            Tx += ry * qz - rz * qy;
            Ty += rz * qx - rx * qz;
            Tz += rx * qy - ry * qx;
        }
    }
    const unsigned full = 0xffffffffu;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        Fx += __shfl_xor_sync(full, Fx, o);
        Fy += __shfl_xor_sync(full, Fy, o);
        Fz += __shfl_xor_sync(full, Fz, o);
        Tx += __shfl_xor_sync(full, Tx, o);
        Ty += __shfl_xor_sync(full, Ty, o);
        Tz += __shfl_xor_sync(full, Tz, o);
    }
    if ((threadIdx.x & 31) == 0) {
        double* F = P.Fh + 3 * p;
        double* T = P.Th + 3 * p;
        atomicAdd(F + 0, (double)Fx);
        atomicAdd(F + 1, (double)Fy);
        atomicAdd(F + 2, (double)Fz);
        atomicAdd(T + 0, (double)Tx);
        atomicAdd(T + 1, (double)Ty);
        atomicAdd(T + 2, (double)Tz);
    }
}

void launch_links(const Lat& L, const PartView& P, const LinkLists& B, cudaStream_t s) {
    if (B.nwarps == 0) return;
    uint64_t threads = (uint64_t)B.nwarps * 32;
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
        for (int a = 0; a < 3; ++a) {
            A.P.Fh[3 * k + a] = 0.0;
            A.P.Th[3 * k + a] = 0.0;
        }
    }
    if (k >= A.band.n) return;
    const Lat& L = A.L;
    int x, y, z;
    unpack_coord(A.band.coord[k], x, y, z);
    int4 cand = A.band.cand[k];
    int c4[4] = {cand.x, cand.y, cand.z, cand.w};
    int best = OWNER_FLUID;
    double best_ratio = 0.0;
    if (L.px || (x > 0 && x < L.nx - 1)) {
        for (int a = 0; a < 4; ++a) {  // candidates ascend, so ties keep the lowest index
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
__global__ void k_map_gather_convert(MapArgs A) {
    uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    uint32_t nf = min(A.st->nflip[A.par], A.F.cap);
    if (w >= nf) return;
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

__global__ void k_map_commit(MapArgs A) {
    uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t nf = min(A.st->nflip[A.par], A.F.cap);
    if (k >= nf) return;
    if (k == 0) atomicAdd(&A.st->flips_total, (unsigned long long)nf);
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

__global__ void k_map_scatter(MapArgs A) {
    uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    uint32_t nf = min(A.st->nflip[A.par], A.F.cap);
    if (w >= nf || lane >= Q) return;
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
    // the queued count is read on the device; grids cover the capacity in
    // warps but exit at once past the count
    uint32_t cap_warps = F.cap;
    uint32_t gblocks = (cap_warps * 32 + 255) / 256;
    // launch only as many blocks as could be needed for a typical step is
    // not possible without a host read; the early exit keeps idle blocks cheap
    k_map_gather_convert<<<gblocks, 256, 0, s>>>(A);
    k_map_commit<<<(F.cap + 255) / 256, 256, 0, s>>>(A);
    k_map_scatter<<<gblocks, 256, 0, s>>>(A);
}

}  // namespace lbmdem
