// lattice.cu -- fluid kernels on the compact AA lattice:
//   * collide+stream, even and odd parity (Section 2.1, Eqs. 4-8), with the
//     probe-plane density and the FP64 mass/momentum totals fused in;
//   * pressure inlet with the oscillating density and the outlet
//     (Section 2.4, Eq. 25, Table 2);
//   * read-out of rho and u (Eq. 7) for any parity.
// Populations are stored as deviations g = f - w rho_f; every formula below is
// the paper's written in g (the weights sum to one, and sum_m w_m c_m = 0).
#include "common.cuh"
#include "kernels.cuh"

namespace lbmdem {

static_assert(cx(opp(7)) == -cx(7) && cy(opp(7)) == -cy(7), "opp");

// Four consecutive populations of one plane (the even kernel's vector
// access): 16 B for FP32, 8 B for the 16-bit forms, streamed (evict-first).
template <int ST> __device__ __forceinline__ float4 ld4(const typename PopT<ST>::T* p, float fsi);
template <> __device__ __forceinline__ float4 ld4<0>(const float* p, float) {
    return __ldcs(reinterpret_cast<const float4*>(p));
}
template <> __device__ __forceinline__ float4 ld4<1>(const __nv_bfloat16* p, float fsi) {
    uint2 r = __ldcs(reinterpret_cast<const uint2*>(p));
    float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&r.x));
    float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&r.y));
    return make_float4(a.x * fsi, a.y * fsi, b.x * fsi, b.y * fsi);
}
template <> __device__ __forceinline__ float4 ld4<2>(const __half* p, float fsi) {
    uint2 r = __ldcs(reinterpret_cast<const uint2*>(p));
    float2 a = __half22float2(*reinterpret_cast<const __half2*>(&r.x));
    float2 b = __half22float2(*reinterpret_cast<const __half2*>(&r.y));
    return make_float4(a.x * fsi, a.y * fsi, b.x * fsi, b.y * fsi);
}
template <int ST> __device__ __forceinline__ void st4(typename PopT<ST>::T* p, float4 v, float fs);
template <> __device__ __forceinline__ void st4<0>(float* p, float4 v, float) {
    __stcs(reinterpret_cast<float4*>(p), v);
}
template <> __device__ __forceinline__ void st4<1>(__nv_bfloat16* p, float4 v, float fs) {
    __nv_bfloat162 a = __floats2bfloat162_rn(v.x * fs, v.y * fs), b = __floats2bfloat162_rn(v.z * fs, v.w * fs);
    uint2 r;
    r.x = *reinterpret_cast<const uint32_t*>(&a);
    r.y = *reinterpret_cast<const uint32_t*>(&b);
    __stcs(reinterpret_cast<uint2*>(p), r);
}
template <> __device__ __forceinline__ void st4<2>(__half* p, float4 v, float fs) {
    __half2 a = __floats2half2_rn(v.x * fs, v.y * fs), b = __floats2half2_rn(v.z * fs, v.w * fs);
    uint2 r;
    r.x = *reinterpret_cast<const uint32_t*>(&a);
    r.y = *reinterpret_cast<const uint32_t*>(&b);
    __stcs(reinterpret_cast<uint2*>(p), r);
}

// Eq. 4 with the equilibrium of Eq. 6 and the moments of Eq. 7, on deviations.
// Returns the moments of the pre-collision state.
__device__ __forceinline__ void bgk(float g[Q], float tau_inv, float rho_f, float& drho, float& jx,
                                    float& jy, float& jz) {
    drho = 0.f;
    jx = jy = jz = 0.f;
#pragma unroll
    for (int m = 0; m < Q; ++m) {
        drho += g[m];
        if (cx(m)) jx += cx(m) > 0 ? g[m] : -g[m];
        if (cy(m)) jy += cy(m) > 0 ? g[m] : -g[m];
        if (cz(m)) jz += cz(m) > 0 ? g[m] : -g[m];
    }
    float rho = rho_f + drho;
    float ir = 1.0f / rho;
    float ux = jx * ir, uy = jy * ir, uz = jz * ir;
    float uu15 = 1.5f * (ux * ux + uy * uy + uz * uz);
    float om = 1.0f - tau_inv;
#pragma unroll
    for (int m = 0; m < Q; ++m) {
        float cu = (float)cx(m) * ux + (float)cy(m) * uy + (float)cz(m) * uz;
        float geq = wt(m) * (drho + rho * (3.0f * cu + 4.5f * cu * cu - uu15));
        g[m] = om * g[m] + tau_inv * geq;
    }
}

struct MonAcc {
    float drho, jx, jy, jz, umax2, cnt;
    float pdrho, pcnt;  // probe plane
    int bad;
};

__device__ __forceinline__ void mon_add(MonAcc& a, float drho, float jx, float jy, float jz,
                                        float rho_f) {
    a.drho += drho;
    a.cnt += 1.f;
    a.jx += jx;
    a.jy += jy;
    a.jz += jz;
    float ir = 1.0f / (rho_f + drho);
    float u2 = (jx * jx + jy * jy + jz * jz) * ir * ir;
    a.umax2 = fmaxf(a.umax2, u2);
    if (!(drho == drho) || !(u2 == u2)) a.bad = 1;
}

// Warp + block reduction of the monitors, one FP64 atomic per block per
// quantity; the probe sums use warp-aggregated atomics.
template <bool MON>
__device__ __forceinline__ void mon_flush(const MonAcc& a, const Mon& mon, bool probe_any) {
    const unsigned full = 0xffffffffu;
    if (mon.probe_sum != nullptr) {
        if (__any_sync(full, a.pcnt > 0.f)) {
            float s = a.pdrho, c = a.pcnt;
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                s += __shfl_xor_sync(full, s, o);
                c += __shfl_xor_sync(full, c, o);
            }
            if ((threadIdx.x & 31) == 0) {
                unsigned long long t = *mon.t_dev - 1ull;  // the map update counted this step
                atomicAdd(&mon.probe_sum[2 * t], (double)s);
                atomicAdd(&mon.probe_sum[2 * t + 1], (double)c);
            }
        }
    }
    if (!MON) return;
    __shared__ double sh[6][32];
    double v[5] = {a.drho, a.jx, a.jy, a.jz, a.cnt};
    float um = a.umax2;
    int bad = a.bad;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
#pragma unroll
        for (int k = 0; k < 5; ++k) v[k] += __shfl_xor_sync(full, v[k], o);
        um = fmaxf(um, __shfl_xor_sync(full, um, o));
        bad |= __shfl_xor_sync(full, bad, o);
    }
    int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        for (int k = 0; k < 5; ++k) sh[k][wid] = v[k];
        sh[5][wid] = (double)um;
        if (bad) atomicOr(mon.status, ST_UNSTABLE);
    }
    __syncthreads();
    if (wid == 0) {
        int nw = blockDim.x >> 5;
        double r[6];
        for (int k = 0; k < 6; ++k) r[k] = lane < nw ? sh[k][lane] : 0.0;
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            for (int k = 0; k < 5; ++k) r[k] += __shfl_xor_sync(full, r[k], o);
            r[5] = fmax(r[5], __shfl_xor_sync(full, r[5], o));
        }
        if (lane == 0) {
            for (int k = 0; k < 5; ++k) atomicAdd(&mon.acc[k], r[k]);
            atomicMax(mon.umax_bits, __float_as_uint((float)r[5]));
        }
    }
}

// Even step: node-local.  Each thread owns 4 consecutive compact nodes and
// moves them with 128-bit loads and stores; solid nodes inside a quad are
// processed harmlessly (their slots are never read while they are solid).
template <bool MON, int ST>
__global__ void __launch_bounds__(256) k_collide_even(Lat L, Mon mon) {
    pdl_wait();
    pdl_trigger();
    auto* f = pops<ST>(L);
    uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t i0 = t * 4u;
    MonAcc a = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    bool active = i0 < L.nS;
    uint32_t bits = 0;
    if (active) {
        bits = (L.fbits[i0 >> 5] >> (i0 & 31)) & 0xfu;
        active = bits != 0;
    }
    if (active) {
        float4 v[Q];
#pragma unroll
        for (int m = 0; m < Q; ++m)
            v[m] = ld4<ST>(f + (size_t)m * L.nSpad + i0, L.fsi);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float g[Q];
#pragma unroll
            for (int m = 0; m < Q; ++m) g[m] = (&v[m].x)[k];
            float drho, jx, jy, jz;
            bgk(g, L.tau_inv, L.rho_f, drho, jx, jy, jz);
#pragma unroll
            for (int m = 0; m < Q; ++m) (&v[opp(m)].x)[k] = g[m];
            if ((bits >> k) & 1u) {
                if (MON) mon_add(a, drho, jx, jy, jz, L.rho_f);
                uint32_t i = i0 + k;
                if ((i >= mon.pA0 && i < mon.pA1) || (i >= mon.pB0 && i < mon.pB1)) {
                    a.pdrho += drho;
                    a.pcnt += 1.f;
                }
            }
        }
#pragma unroll
        for (int m = 0; m < Q; ++m)
            st4<ST>(f + (size_t)m * L.nSpad + i0, v[m], L.fs);
    }
    mon_flush<MON>(a, mon, true);
}

// ---- even step with the step's links (one node per lane and 32-node run)
//
// The even step is node-local, so the links of a node can be bounced where
// its post-collision values are written.  For a link direction m of fluid
// node x (x + c_m solid, owned by sphere p) the value leaving towards the
// wall, g~_m, goes to slot opp(m) of x as g~_m - delta (Eq. 14, moving wall),
//     delta = 6 w_m rho_f c_m . U,   U = V + W x r,   r = x - X,
// the wall velocity at x (the half-link offset c_m / 2 drops out because
// c_m . (W x c_m) = 0), and adds the link force c_m (2 g~_m - delta) of
// Eq. 15 (counted about the rest state, as the link kernel does) and its
// torque r x c_m (2 g~_m - delta) of Eq. 19 to the sphere.  Each thread keeps
// two (sphere, force, torque) slots; at the end the warp sums the slots
// sphere by sphere and adds each sum with one FP64 atomic per component.

struct LinkSlot {
    int p;
    float v[6];  // force xyz, torque xyz
};

__device__ __forceinline__ void slot_put(LinkSlot& s, int p, const float v[6]) {
    if (s.p < 0) {
        s.p = p;
#pragma unroll
        for (int c = 0; c < 6; ++c) s.v[c] = v[c];
    } else {
#pragma unroll
        for (int c = 0; c < 6; ++c) s.v[c] += v[c];
    }
}

__device__ __forceinline__ void slot_add(LinkSlot& s0, LinkSlot& s1, const PartView& P, int p, const float v[6],
                                         uint32_t rep) {
    if (s0.p == p || s0.p < 0) {
        slot_put(s0, p, v);
    } else if (s1.p == p || s1.p < 0) {
        slot_put(s1, p, v);
    } else {  // a third sphere: add the second slot to the sums and reuse it
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            atomicAdd(P.Fh + 3 * ((size_t)rep * P.n + s1.p) + c, (double)s1.v[c]);
            atomicAdd(P.Th + 3 * ((size_t)rep * P.n + s1.p) + c, (double)s1.v[c + 3]);
        }
        s1.p = -1;
        slot_put(s1, p, v);
    }
}

// The links of node (x, y, z) to sphere p (bit m of msk: direction m).
__device__ __forceinline__ void node_links(const Lat& L, const PartView& P, int x, int y, int z, int p, uint32_t msk,
                                           float g[Q], float out[6]) {
    const float4 a = P.pk[3 * (size_t)p], b = P.pk[3 * (size_t)p + 1], c = P.pk[3 * (size_t)p + 2];
    const int ox = __float_as_int(c.y), oy = __float_as_int(c.z), oz = __float_as_int(c.w);
    const int ix = L.px ? imin_small(x - ox, L.nx) : x - ox;
    const int iy = imin_small(y - oy, L.ny), iz = imin_small(z - oz, L.nz);
    const float rx = (float)ix - a.x, ry = (float)iy - a.y, rz = (float)iz - a.z;
    const float Ux = a.w + (b.w * rz - c.x * ry), Uy = b.x + (c.x * rx - b.z * rz), Uz = b.y + (b.z * ry - b.w * rx);
    const float s6 = 6.0f * L.rho_f;
    float fx = 0.f, fy = 0.f, fz = 0.f;
#pragma unroll
    for (int m = 0; m < Q - 1; ++m) {
        if (!((msk >> m) & 1u)) continue;
        const float cu = (float)cx(m) * Ux + (float)cy(m) * Uy + (float)cz(m) * Uz;
        const float d = (s6 * wt(m)) * cu;
        const float v = g[m];
        g[m] = v - d;
        const float q = 2.0f * v - d;
        if (cx(m)) fx += cx(m) > 0 ? q : -q;
        if (cy(m)) fy += cy(m) > 0 ? q : -q;
        if (cz(m)) fz += cz(m) > 0 ? q : -q;
    }
    out[0] = fx;
    out[1] = fy;
    out[2] = fz;
    out[3] = ry * fz - rz * fy;
    out[4] = rz * fx - rx * fz;
    out[5] = rx * fy - ry * fx;
}

// owner of the neighbour x + c_m (a link direction, so in range)
__device__ __forceinline__ int neighbour_owner(const Lat& L, int x, int y, int z, int m) {
    int xs = x + cx(m);
    if (L.px) xs = wrap1(xs, L.nx);
    const int ys = wrap1(y + cy(m), L.ny), zs = wrap1(z + cz(m), L.nz);
    return L.owner[((size_t)xs * L.ny + ys) * L.nz + zs];
}

template <int ST> __device__ __forceinline__ float ld1(const typename PopT<ST>::T* p, float fsi) {
    return to_f<ST>(*p, fsi);
}
template <> __device__ __forceinline__ float ld1<0>(const float* p, float) { return __ldcs(p); }
template <int ST> __device__ __forceinline__ void st1(typename PopT<ST>::T* p, float v, float fs) {
    *p = from_f<ST>(v, fs);
}
template <> __device__ __forceinline__ void st1<0>(float* p, float v, float) { __stcs(p, v); }

// Each warp takes EVEN_ROUNDS consecutive runs of 32 nodes, one node per
// lane and run (coalesced); the lanes' sphere slots carry over from run to
// run (neighbouring runs mostly touch the same spheres), so the warp sums
// them once per 32 EVEN_ROUNDS nodes.
constexpr int EVEN_ROUNDS = 2;

// 72 registers (a few spills to L1): 28 resident warps per SM instead of 24
// at the 80 the kernel would otherwise take, which hides more of the
// population loads' latency (187 against 190 us on the 128 x 128 x 1024
// column).  Launched with up to 256 threads per block.
template <bool MON, int ST>
__global__ void __maxnreg__(72) k_collide_even_links(Lat L, Mon mon, PartView P, const uint2* __restrict__ lwp) {
    pdl_wait();
    pdl_trigger();
    auto* f = pops<ST>(L);
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t rep = gw % NREP;
    MonAcc a = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    LinkSlot s0, s1;
    s0.p = s1.p = -1;
#pragma unroll
    for (int c = 0; c < 6; ++c) s0.v[c] = s1.v[c] = 0.f;
    for (int run = 0; run < EVEN_ROUNDS; ++run) {
    const uint32_t i = (gw * EVEN_ROUNDS + run) * 32u + (threadIdx.x & 31);
    if (i < L.nS && fluid_bit(L, i)) {
        float g[Q];
#pragma unroll
        for (int m = 0; m < Q; ++m) g[m] = ld1<ST>(f + (size_t)m * L.nSpad + i, L.fsi);
        const uint2 w = __ldg(&lwp[i]);
        const uint32_t cw = __ldg(&L.coord[i]);
        float drho, jx, jy, jz;
        bgk(g, L.tau_inv, L.rho_f, drho, jx, jy, jz);
        if (MON) mon_add(a, drho, jx, jy, jz, L.rho_f);
        if ((i >= mon.pA0 && i < mon.pA1) || (i >= mon.pB0 && i < mon.pB1)) {
            a.pdrho += drho;
            a.pcnt += 1.f;
        }
        const uint32_t mask = w.x & LW_MASK;
        if (mask) {
            int x, y, z;
            unpack_coord(cw, x, y, z);
            const uint32_t pa = w.x >> 18, pb = w.y >> 18, sel = w.y & LW_MASK;
            float v[6];
            if (pa != LW_NONE) {
                node_links(L, P, x, y, z, (int)pa, mask & ~sel, g, v);
                slot_add(s0, s1, P, (int)pa, v, rep);
                if (sel) {
                    node_links(L, P, x, y, z, (int)pb, sel, g, v);
                    slot_add(s0, s1, P, (int)pb, v, rep);
                }
            } else {
                // neighbours of more than two spheres: one sphere at a time
                uint32_t rem = mask;
                while (rem) {
                    int p = -1;
#pragma unroll
                    for (int m = 0; m < Q - 1; ++m)
                        if (p < 0 && ((rem >> m) & 1u)) p = neighbour_owner(L, x, y, z, m);
                    uint32_t sub = 0u;
#pragma unroll
                    for (int m = 0; m < Q - 1; ++m)
                        if (((rem >> m) & 1u) && neighbour_owner(L, x, y, z, m) == p) sub |= 1u << m;
                    node_links(L, P, x, y, z, p, sub, g, v);
                    slot_add(s0, s1, P, p, v, rep);
                    rem &= ~sub;
                }
            }
        }
#pragma unroll
        for (int m = 0; m < Q; ++m) st1<ST>(f + (size_t)opp(m) * L.nSpad + i, g[m], L.fs);
    }
    }
    // the warp's slots, sphere by sphere: lanes holding the sphere contribute
    const unsigned full = 0xffffffffu;
    const uint32_t lane = threadIdx.x & 31;
    for (;;) {
        const int mine = s0.p >= 0 ? s0.p : s1.p;
        const unsigned act = __ballot_sync(full, mine >= 0);
        if (!act) break;
        const int p = __shfl_sync(full, mine, __ffs(act) - 1);
        float s8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (s0.p == p) {
#pragma unroll
            for (int c = 0; c < 6; ++c) s8[c] += s0.v[c];
            s0.p = -1;
        }
        if (s1.p == p) {
#pragma unroll
            for (int c = 0; c < 6; ++c) s8[c] += s1.v[c];
            s1.p = -1;
        }
        // transposing butterfly (lane l ends with component 4 b4 + 2 b3 + b2)
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
            const size_t r = (size_t)rep * P.n + p;
            double* dst = comp < 3 ? P.Fh + 3 * r + comp : P.Th + 3 * r + (comp - 3);
            atomicAdd(dst, (double)s8[0]);
        }
    }
    mon_flush<MON>(a, mon, true);
}

template <int ST>
static void launch_even_links_st(const Lat& L, const Mon& mon, const PartView& P, const uint2* lw, bool monitor,
                                 int tile, cudaStream_t s) {
    const uint32_t blocks = (L.nS + tile * EVEN_ROUNDS - 1) / (tile * EVEN_ROUNDS);
    if (monitor)
        launch_pdl(k_collide_even_links<true, ST>, blocks, tile, s, L, mon, P, lw);
    else
        launch_pdl(k_collide_even_links<false, ST>, blocks, tile, s, L, mon, P, lw);
}

void launch_collide_even_links(const Lat& L, const Mon& mon, const PartView& P, const uint2* lw, bool monitor,
                               int tile, cudaStream_t s) {
    if (L.nS == 0) return;
    switch (L.st) {
        case 0: launch_even_links_st<0>(L, mon, P, lw, monitor, tile, s); break;
        case 1: launch_even_links_st<1>(L, mon, P, lw, monitor, tile, s); break;
        default: launch_even_links_st<2>(L, mon, P, lw, monitor, tile, s); break;
    }
}

// compact index of bit `bit` of a word record if that node is fluid now
__device__ __forceinline__ uint32_t word_index(const uint4& r, const uint32_t* mBp, uint32_t bit) {
    if (!(r.x & bit)) return NONE;
    uint32_t low = bit - 1u;
    if (r.y & bit) return r.z + __popc(r.y & low);
    return r.w + __popc(__ldg(mBp) & low);
}

// Neighbours x + c_m of node (x, y, z) on the z-line (xs, ys): the record of
// the word holding z serves dz = -1, 0, +1 unless z +- 1 crosses a word.
struct LineProbe {
    const Lat& L;
    size_t wl;
    int w0;
    uint4 r0;
    __device__ __forceinline__ LineProbe(const Lat& L_, int xs, int ys, int z) : L(L_) {
        wl = ((size_t)xs * L.ny + ys) * L.nw;
        w0 = z >> 5;
        r0 = __ldg(&L.rec[wl + w0]);
    }
    __device__ __forceinline__ uint32_t at(int zs) const {
        int wz = zs >> 5;
        uint4 r = wz == w0 ? r0 : __ldg(&L.rec[wl + wz]);
        return word_index(r, &L.maskB[wl + wz], 1u << (zs & 31));
    }
};

// Odd step: node x gathers direction m from slot opp(m) of x - c_m (or from
// its own slot m when x - c_m is solid or outside), collides, and scatters
// direction m to slot m of x + c_m (or its own slot opp(m)).  Each thread
// reads and writes the same 19 locations, so the update is in place.
template <bool MON, int ST>
__global__ void __launch_bounds__(256, 4) k_collide_odd(Lat L, Mon mon) {
    pdl_wait();
    pdl_trigger();
    auto* f = pops<ST>(L);
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    MonAcc a = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    bool active = i < L.nS && fluid_bit(L, i);
    if (active) {
        int x, y, z;
        unpack_coord(__ldcs(&L.coord[i]), x, y, z);
        const int zm = z == 0 ? L.nz - 1 : z - 1, zp = z == L.nz - 1 ? 0 : z + 1;
        const int ym = y == 0 ? L.ny - 1 : y - 1, yp = y == L.ny - 1 ? 0 : y + 1;
        int xm = x - 1, xp = x + 1;
        bool hasm = true, hasp = true;
        if (L.px) {
            xm = x == 0 ? L.nx - 1 : xm;
            xp = x == L.nx - 1 ? 0 : xp;
        } else {
            hasm = x > 0;
            hasp = x < L.nx - 1;
        }
        uint32_t nb[Q - 1];  // compact index of x + c_m, or NONE
        {
            LineProbe l(L, x, y, z);
            nb[4] = l.at(zp);
            nb[5] = l.at(zm);
        }
        {
            LineProbe l(L, x, yp, z);
            nb[2] = l.at(z);
            nb[14] = l.at(zp);
            nb[15] = l.at(zm);
        }
        {
            LineProbe l(L, x, ym, z);
            nb[3] = l.at(z);
            nb[16] = l.at(zp);
            nb[17] = l.at(zm);
        }
        if (hasp) {
            {
                LineProbe l(L, xp, y, z);
                nb[0] = l.at(z);
                nb[8] = l.at(zp);
                nb[9] = l.at(zm);
            }
            nb[6] = LineProbe(L, xp, yp, z).at(z);
            nb[7] = LineProbe(L, xp, ym, z).at(z);
        } else {
            nb[0] = nb[8] = nb[9] = nb[6] = nb[7] = NONE;
        }
        if (hasm) {
            {
                LineProbe l(L, xm, y, z);
                nb[1] = l.at(z);
                nb[12] = l.at(zp);
                nb[13] = l.at(zm);
            }
            nb[10] = LineProbe(L, xm, yp, z).at(z);
            nb[11] = LineProbe(L, xm, ym, z).at(z);
        } else {
            nb[1] = nb[12] = nb[13] = nb[10] = nb[11] = NONE;
        }
        // 32-bit element offsets (19 nSpad < 2^32, checked at the layout)
        float g[Q];
#pragma unroll
        for (int m = 0; m < Q - 1; ++m) {
            uint32_t s = nb[opp(m)];
            const uint32_t off = s != NONE ? (uint32_t)opp(m) * L.nSpad + s : (uint32_t)m * L.nSpad + i;
            g[m] = to_f<ST>(f[off], L.fsi);
        }
        g[18] = to_f<ST>(f[18u * L.nSpad + i], L.fsi);
        float drho, jx, jy, jz;
        bgk(g, L.tau_inv, L.rho_f, drho, jx, jy, jz);
#pragma unroll
        for (int m = 0; m < Q - 1; ++m) {
            uint32_t d = nb[m];
            const uint32_t off = d != NONE ? (uint32_t)m * L.nSpad + d : (uint32_t)opp(m) * L.nSpad + i;
            f[off] = from_f<ST>(g[m], L.fs);
        }
        f[18u * L.nSpad + i] = from_f<ST>(g[18], L.fs);
        if (MON) mon_add(a, drho, jx, jy, jz, L.rho_f);
        if ((i >= mon.pA0 && i < mon.pA1) || (i >= mon.pB0 && i < mon.pB1)) {
            a.pdrho += drho;
            a.pcnt += 1.f;
        }
    }
    mon_flush<MON>(a, mon, true);
}

template <int ST>
static void launch_collide_st(const Lat& L, const Mon& mon, bool odd, bool monitor, int tile, cudaStream_t s) {
    if (!odd) {
        uint32_t threads = (L.nS + 3) / 4;
        uint32_t blocks = (threads + tile - 1) / tile;
        if (monitor)
            launch_pdl(k_collide_even<true, ST>, blocks, tile, s, L, mon);
        else
            launch_pdl(k_collide_even<false, ST>, blocks, tile, s, L, mon);
    } else {
        uint32_t blocks = (L.nS + tile - 1) / tile;
        if (monitor)
            launch_pdl(k_collide_odd<true, ST>, blocks, tile, s, L, mon);
        else
            launch_pdl(k_collide_odd<false, ST>, blocks, tile, s, L, mon);
    }
}

// tile: threads per block (64, 128 or 256; the kernels are bounded for 256)
void launch_collide(const Lat& L, const Mon& mon, bool odd, bool monitor, int tile, cudaStream_t s) {
    if (L.nS == 0) return;
    switch (L.st) {
        case 0: launch_collide_st<0>(L, mon, odd, monitor, tile, s); break;
        case 1: launch_collide_st<1>(L, mon, odd, monitor, tile, s); break;
        default: launch_collide_st<2>(L, mon, odd, monitor, tile, s); break;
    }
}

// ------------------------------------------------------------ inlet / outlet

template <bool AFTER_EVEN, int ST>
__global__ void k_inlet_outlet(Lat L, BC bc) {
    auto* f = pops<ST>(L);
    __shared__ float s_drho;
    // the density the step ends with: t + 1, counted by the map update
    if (threadIdx.x == 0) s_drho = (float)source_drho(bc.src, *bc.t_dev);
    __syncthreads();
    int plane = L.ny * L.nz;
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 2 * plane) return;
    int side = k >= plane;
    int yz = side ? k - plane : k;
    int y = yz / L.nz, z = yz - y * L.nz;
    int x = side ? L.nx - 1 : 0;
    bool fl;
    uint32_t i = stored_index(L, x, y, z, fl);
    if (!fl || i == NONE) return;
    if (side == 0) {
        if (bc.inlet != 0) return;
        float g[Q];
#pragma unroll
        for (int m = 0; m < Q; ++m)
            if (cx(m) <= 0) g[m] = to_f<ST>(*pop_loc<ST>(L, AFTER_EVEN, x, y, z, i, m), L.fsi);
        pressure_face(g, s_drho, 0);
#pragma unroll
        for (int m = 0; m < Q; ++m)
            if (cx(m) > 0) f[(size_t)m * L.nSpad + i] = from_f<ST>(g[m], L.fs);  // source outside: own slot
    } else if (bc.outlet == 0) {
        bool ufl;
        uint32_t u = stored_index(L, x - 1, y, z, ufl);
        if (!ufl || u == NONE) return;
#pragma unroll
        for (int m = 0; m < Q; ++m)
            if (cx(m) < 0) f[(size_t)m * L.nSpad + i] = *pop_loc<ST>(L, AFTER_EVEN, x - 1, y, z, u, m);
    } else if (bc.outlet == 1) {
        float g[Q];
#pragma unroll
        for (int m = 0; m < Q; ++m)
            if (cx(m) >= 0) g[m] = to_f<ST>(*pop_loc<ST>(L, AFTER_EVEN, x, y, z, i, m), L.fsi);
        pressure_face(g, 0.f, 1);
#pragma unroll
        for (int m = 0; m < Q; ++m)
            if (cx(m) < 0) f[(size_t)m * L.nSpad + i] = from_f<ST>(g[m], L.fs);
    }
}

void launch_inlet_outlet(const Lat& L, const BC& bc, bool after_even, cudaStream_t s) {
    if (L.px) return;
    if (bc.inlet != 0 && bc.outlet > 1) return;
    int n = 2 * L.ny * L.nz;
    int blocks = (n + 127) / 128;
#define LBMDEM_IO(AE, ST) k_inlet_outlet<AE, ST><<<blocks, 128, 0, s>>>(L, bc)
    if (after_even) {
        if (L.st == 0) LBMDEM_IO(true, 0);
        else if (L.st == 1) LBMDEM_IO(true, 1);
        else LBMDEM_IO(true, 2);
    } else {
        if (L.st == 0) LBMDEM_IO(false, 0);
        else if (L.st == 1) LBMDEM_IO(false, 1);
        else LBMDEM_IO(false, 2);
    }
#undef LBMDEM_IO
}

// ------------------------------------------------------------ read-out

template <int ST>
__global__ void k_read_fields(Lat L, bool after_even, double* rho, double* u, uint8_t* solid) {
    size_t N = (size_t)L.nx * L.ny * L.nz;
    size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    int z = (int)(n % L.nz);
    size_t r = n / L.nz;
    int y = (int)(r % L.ny);
    int x = (int)(r / L.ny);
    bool fl;
    uint32_t i = stored_index(L, x, y, z, fl);
    fl = fl && i != NONE;
    if (solid) solid[n] = fl ? 0 : 1;
    double d = 0, jx = 0, jy = 0, jz = 0;
    if (fl) {
#pragma unroll
        for (int m = 0; m < Q; ++m) {
            double g = (double)to_f<ST>(*pop_loc<ST>(L, after_even, x, y, z, i, m), L.fsi);
            d += g;
            jx += cx(m) * g;
            jy += cy(m) * g;
            jz += cz(m) * g;
        }
    }
    double rr = fl ? (double)L.rho_f + d : 0.0;
    if (rho) rho[n] = rr;
    if (u) {
        u[n] = fl ? jx / rr : 0.0;
        u[N + n] = fl ? jy / rr : 0.0;
        u[2 * N + n] = fl ? jz / rr : 0.0;
    }
}

void launch_read_fields(const Lat& L, bool after_even, double* rho, double* u, uint8_t* solid,
                        cudaStream_t s) {
    size_t N = (size_t)L.nx * L.ny * L.nz;
    unsigned blocks = (unsigned)((N + 255) / 256);
    if (L.st == 0) k_read_fields<0><<<blocks, 256, 0, s>>>(L, after_even, rho, u, solid);
    else if (L.st == 1) k_read_fields<1><<<blocks, 256, 0, s>>>(L, after_even, rho, u, solid);
    else k_read_fields<2><<<blocks, 256, 0, s>>>(L, after_even, rho, u, solid);
}

// ------------------------------------------------------------ plane means

// Sums over the fluid nodes of every x plane of the current state: out[3 x]
// += sum (rho - rho_f), out[3 x + 1] += sum rho u_x, out[3 x + 2] += count.
// Consecutive compact nodes share a plane, so each warp reduces runs of
// equal x before one FP64 atomic per run head.
template <int ST>
__global__ void k_plane_sums(Lat L, bool after_even, double* out) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    float d = 0.f, jx = 0.f, n = 0.f;
    int x = -1;
    if (i < L.nS && fluid_bit(L, i)) {
        int y, z;
        unpack_coord(L.coord[i], x, y, z);
#pragma unroll
        for (int m = 0; m < Q; ++m) {
            float g = to_f<ST>(*pop_loc<ST>(L, after_even, x, y, z, i, m), L.fsi);
            d += g;
            jx += cx(m) * g;
        }
        n = 1.f;
    }
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    // sums over the lanes of the warp that share this lane's plane; the
    // lowest such lane adds them (compact order keeps most warps in one plane)
    double sd = 0.0, sj = 0.0, sn = 0.0;
    for (int l = 0; l < 32; ++l) {
        float a = __shfl_sync(full, d, l), b = __shfl_sync(full, jx, l), c = __shfl_sync(full, n, l);
        int xl = __shfl_sync(full, x, l);
        if (xl == x) {
            sd += a;
            sj += b;
            sn += c;
        }
    }
    unsigned peers = __match_any_sync(full, x);
    if (x >= 0 && lane == __ffs(peers) - 1) {
        atomicAdd(&out[3 * x], sd);
        atomicAdd(&out[3 * x + 1], sj);
        atomicAdd(&out[3 * x + 2], sn);
    }
}

void launch_plane_sums(const Lat& L, bool after_even, double* out, cudaStream_t s) {
    unsigned blocks = (L.nS + 255) / 256;
    if (!blocks) return;
    if (L.st == 0) k_plane_sums<0><<<blocks, 256, 0, s>>>(L, after_even, out);
    else if (L.st == 1) k_plane_sums<1><<<blocks, 256, 0, s>>>(L, after_even, out);
    else k_plane_sums<2><<<blocks, 256, 0, s>>>(L, after_even, out);
}

}  // namespace lbmdem
