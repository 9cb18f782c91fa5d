// dem.cu -- the solid phase (Section 2.2, Eqs. 9-12).
//
//  * k_dem_step_dsm: one launch per LBM step, one thread-block cluster of up
//    to 16 CTAs, a team of TEAM threads per sphere holding the sphere's
//    state in registers; positions and half-step velocities are exchanged
//    through distributed shared memory.  k_dem_step is the general form
//    (state in global memory, several spheres per team) for packings too
//    large for one cluster, and computes the initial contact forces.
//  * Both: one thread-block cluster (co-scheduled), a team per sphere.  It runs the K velocity-
//    Verlet substeps of length 1/K with the hydrodynamic force and torque of
//    the step held fixed: kick + drift of the own sphere, one cluster barrier,
//    then the contact forces of the own sphere from its neighbour list and
//    the closing kick.  Positions and half-step velocities read by the
//    neighbours are double-buffered by substep parity, so one barrier per
//    substep suffices.  Each pair is evaluated by both spheres with mirror-
//    exact arithmetic, so the two forces are exact negatives and no atomics
//    are needed.  The hydrodynamic force and torque that drive a sphere are
//    the mean of the exchange sums of this and the previous LBM step (the
//    half-way bounce-back force alternates from step to step; the two-step
//    mean of Ladd's momentum-exchange method keeps the explicit coupling of
//    light spheres stable).
//  * neighbour lists: uniform cells of size >= 2 R_max + skin over the
//    periodic y, z box; every periodic image is a separate entry (a sphere in
//    a narrow box can touch two images of the same neighbour).  Rebuilt only
//    at re-layouts; the tangential history is carried over by (j, image).
//
// Positions are X = Xref (FP64, fixed between re-layouts) + dX (FP32 with a
// Kahan compensation term), so the substep loop needs no FP64 arithmetic.
#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"
#include "layout.cuh"

namespace cg = cooperative_groups;

namespace lbmdem {

__device__ __forceinline__ float3 f3(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float3 crossf(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

constexpr int TEAM = 4;  // threads per sphere: they share its neighbour list

// One contact of sphere i with neighbour entry (j, image) (Eqs. 11-12):
// Hertz normal force, incremental Mindlin tangential force from the
// half-step relative velocity at the contact point, previous tangential
// force projected on the current tangent plane, Coulomb cap.  dl = dX_j -
// dX_i; dr = the entry's reference separation (w: (R_i + R_j)^2 - |xyz|^2).
// Updates the history h (force on i) and adds the force and torque on i.
// The arithmetic is mirror-exact: sphere j, evaluating the same pair,
// obtains exactly the negative force.  Square roots and divisions use the
// hardware approximations (reciprocal square root, fast divide; a few ulp):
// deterministic functions of symmetric operands, so exactness of the pair
// is kept.
__device__ __forceinline__ void pair_contact(const Dem& D, float Ri, float Rj, float3 dl, float4 dr, float3 vi,
                                             float3 wi, float3 vj, float3 wj, float dt_inc, float4& h, float3& F,
                                             float3& T) {
    float3 d = make_float3(dr.x + dl.x, dr.y + dl.y, dr.z + dl.z);
    float cut = Ri + Rj;
    // cut^2 - |d|^2 without cancellation: e0 - 2 dref.dl - dl.dl
    float qd = dr.w - (2.f * (dr.x * dl.x + dr.y * dl.y + dr.z * dl.z) + (dl.x * dl.x + dl.y * dl.y + dl.z * dl.z));
    if (!(qd > 0.f)) {
        h = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    float d2 = d.x * d.x + d.y * d.y + d.z * d.z;
    float idist = rsqrtf(d2);
    float dist = d2 * idist;
    float delta = __fdividef(qd, cut + dist);
    float3 n = make_float3(d.x * idist, d.y * idist, d.z * idist);
    float Rs = __fdividef(Ri * Rj, Ri + Rj);
    float rd = Rs * delta;
    float sq = rd * rsqrtf(rd);
    float fn = D.kn * sq * delta;
    float ai = Ri - 0.5f * delta, aj = Rj - 0.5f * delta;
    float3 ri = make_float3(ai * n.x, ai * n.y, ai * n.z);
    float3 rj = make_float3(-(aj * n.x), -(aj * n.y), -(aj * n.z));
    float3 cwj = crossf(wj, rj), cwi = crossf(wi, ri);
    float3 vr = make_float3((vj.x + cwj.x) - (vi.x + cwi.x), (vj.y + cwj.y) - (vi.y + cwi.y),
                            (vj.z + cwj.z) - (vi.z + cwi.z));
    float vn = vr.x * n.x + vr.y * n.y + vr.z * n.z;
    float3 vt = make_float3(vr.x - vn * n.x, vr.y - vn * n.y, vr.z - vn * n.z);
    float hn = h.x * n.x + h.y * n.y + h.z * n.z;
    float kdt = D.kt * sq * dt_inc;
    float3 ft = make_float3(h.x - hn * n.x + kdt * vt.x, h.y - hn * n.y + kdt * vt.y, h.z - hn * n.z + kdt * vt.z);
    float ftm2 = ft.x * ft.x + ft.y * ft.y + ft.z * ft.z;
    float cap = D.mu * fn;
    if (ftm2 > cap * cap) {  // |F_t| > mu |F_n|, compared in squares
        float sc = cap * rsqrtf(ftm2);
        ft = make_float3(ft.x * sc, ft.y * sc, ft.z * sc);
    }
    h = make_float4(ft.x, ft.y, ft.z, 0.f);
    float3 Fk = make_float3(-fn * n.x + ft.x, -fn * n.y + ft.y, -fn * n.z + ft.z);
    float3 Tk = crossf(ri, Fk);
    F.x += Fk.x;
    F.y += Fk.y;
    F.z += Fk.z;
    T.x += Tk.x;
    T.y += Tk.y;
    T.z += Tk.z;
}

// Contact forces on sphere i from its neighbour list, positions and half-
// step velocities of substep buffer b in global memory.  dt_inc = 0
// evaluates without tangential increment.  Lane `tl` of the sphere's team
// takes entries tl, tl + TEAM, ...; the caller reduces over the team.
__device__ void contact_forces(const Dem& D, int i, int b, float dt_inc, int tl, float3& F, float3& T) {
    F = make_float3(0.f, 0.f, 0.f);
    T = make_float3(0.f, 0.f, 0.f);
    float3 xi = f3(__ldcg(&D.dXb[b * D.n + i]));
    float3 vi = f3(__ldcg(&D.Vhb[b * D.n + i])), wi = f3(__ldcg(&D.Whb[b * D.n + i]));
    float Ri = D.R[i];
    int cnt = D.nb_cnt[i];
    for (int k = tl; k < cnt; k += TEAM) {
        size_t e = (size_t)i * D.nbmax + k;
        int j = D.nb_j[e];
        float4 dr = D.nb_dref[e];
        float3 xj = f3(__ldcg(&D.dXb[b * D.n + j]));
        float3 vj = f3(__ldcg(&D.Vhb[b * D.n + j])), wj = f3(__ldcg(&D.Whb[b * D.n + j]));
        float4 h = D.nb_ft[e];
        pair_contact(D, Ri, D.R[j], make_float3(xj.x - xi.x, xj.y - xi.y, xj.z - xi.z), dr, vi, wi, vj, wj,
                     dt_inc, h, F, T);
        D.nb_ft[e] = h;
    }
}

// First half kick of velocity Verlet and the drift of one substep:
// half-step velocities vh, wh from the contact (fc, tc), hydrodynamic (fa,
// ta) and body forces; the displacement dx advanced with Kahan-compensated
// FP32 accumulation (compensation c); q <- normalize(q + dt/2 (0, wh) q).
__device__ __forceinline__ void kick_drift(const Dem& D, float3 fc, float3 tc, float3 fa, float3 ta, float im,
                                           float iI, float3 v, float3 w, float3& vh, float3& wh, float3& dx,
                                           float3& c, float4& q) {
    const float dt = D.dt;
    vh = make_float3(v.x + 0.5f * dt * (fc.x + fa.x + D.g.x) * im, v.y + 0.5f * dt * (fc.y + fa.y + D.g.y) * im,
                     v.z + 0.5f * dt * (fc.z + fa.z + D.g.z) * im);
    wh = make_float3(w.x + 0.5f * dt * (tc.x + ta.x) * iI, w.y + 0.5f * dt * (tc.y + ta.y) * iI,
                     w.z + 0.5f * dt * (tc.z + ta.z) * iI);
    float yx = dt * vh.x - c.x, yy = dt * vh.y - c.y, yz = dt * vh.z - c.z;
    float tx = dx.x + yx, ty = dx.y + yy, tz = dx.z + yz;
    c = make_float3((tx - dx.x) - yx, (ty - dx.y) - yy, (tz - dx.z) - yz);
    dx = make_float3(tx, ty, tz);
    float dq0 = -(wh.x * q.y + wh.y * q.z + wh.z * q.w);
    float3 wxv = crossf(wh, make_float3(q.y, q.z, q.w));
    float4 dq = make_float4(dq0, q.x * wh.x + wxv.x, q.x * wh.y + wxv.y, q.x * wh.z + wxv.z);
    q = make_float4(q.x + 0.5f * dt * dq.x, q.y + 0.5f * dt * dq.y, q.z + 0.5f * dt * dq.z, q.w + 0.5f * dt * dq.w);
    float nq = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    q = make_float4(q.x * nq, q.y * nq, q.z * nq, q.w * nq);
}

// Second half kick: V = vh + dt/2 (F + fa + g) / m, W likewise.
__device__ __forceinline__ void close_kick(const Dem& D, float3 vh, float3 wh, float3 F, float3 T, float3 fa,
                                           float3 ta, float im, float iI, float3& v, float3& w) {
    const float dt = D.dt;
    v = make_float3(vh.x + 0.5f * dt * (F.x + fa.x + D.g.x) * im, vh.y + 0.5f * dt * (F.y + fa.y + D.g.y) * im,
                    vh.z + 0.5f * dt * (F.z + fa.z + D.g.z) * im);
    w = make_float3(wh.x + 0.5f * dt * (T.x + ta.x) * iI, wh.y + 0.5f * dt * (T.y + ta.y) * iI,
                    wh.z + 0.5f * dt * (T.z + ta.z) * iI);
}

// sum over the TEAM lanes of a sphere (lanes of a team are consecutive)
__device__ __forceinline__ void team_sum(float3& F, float3& T) {
    const unsigned full = 0xffffffffu;
#pragma unroll
    for (int o = 1; o < TEAM; o <<= 1) {
        F.x += __shfl_xor_sync(full, F.x, o);
        F.y += __shfl_xor_sync(full, F.y, o);
        F.z += __shfl_xor_sync(full, F.z, o);
        T.x += __shfl_xor_sync(full, T.x, o);
        T.y += __shfl_xor_sync(full, T.y, o);
        T.z += __shfl_xor_sync(full, T.z, o);
    }
}

// Lattice frame of sphere i after the step (integer origin, wrapped origin,
// FP32 offset of the centre) and its displacement / speed for the
// re-layout decision and the NaN / skin checks.
__device__ __forceinline__ void sphere_frame(const Dem& D, int i, float& dmax, float& vmax, uint32_t& bad) {
    float4 dx = D.dX[i], c = D.dXc[i], v = D.V[i];
    double X0 = D.Xref[3 * i] + (double)dx.x - (double)c.x;
    double X1 = D.Xref[3 * i + 1] + (double)dx.y - (double)c.y;
    double X2 = D.Xref[3 * i + 2] + (double)dx.z - (double)c.z;
    int4 o = make_int4((int)floor(D.Xref[3 * i]), (int)floor(D.Xref[3 * i + 1]), (int)floor(D.Xref[3 * i + 2]), 0);
    D.org[i] = o;
    int wx = D.px ? (int)(((long long)o.x % (long long)D.Lx + (long long)D.Lx) % (long long)D.Lx) : o.x;
    int wy = (int)(((long long)o.y % (long long)D.Ly + (long long)D.Ly) % (long long)D.Ly);
    int wz = (int)(((long long)o.z % (long long)D.Lz + (long long)D.Lz) % (long long)D.Lz);
    D.orgw[i] = make_int4(wx, wy, wz, 0);
    D.xf[i] = make_float4((float)(X0 - o.x), (float)(X1 - o.y), (float)(X2 - o.z), 0.f);
    float dd = sqrtf(dx.x * dx.x + dx.y * dx.y + dx.z * dx.z);
    float vv = sqrtf(v.x * v.x + v.y * v.y + v.z * v.z);
    if (!(dd == dd) || !(vv == vv) || isinf(dd) || isinf(vv)) bad |= ST_UNSTABLE;
    else if (dd >= D.hard_disp) bad |= ST_SKIN;
    dmax = fmaxf(dmax, dd);
    vmax = fmaxf(vmax, vv);
}

// The same outputs for the per-step kernel: the integer origins depend only
// on Xref, which changes only at re-layouts (after which the general kernel
// runs sphere_frame), so only the FP32 offset of the centre is renewed.
// Lane `tl` < 3 of the sphere's team computes axis tl; lane 0 checks.
__device__ __forceinline__ void sphere_offset(const Dem& D, int i, int tl, float& dmax, float& vmax, uint32_t& bad) {
    if (tl < 3) {
        const float* dx = reinterpret_cast<const float*>(&D.dX[i]);
        const float* c = reinterpret_cast<const float*>(&D.dXc[i]);
        const int* o = reinterpret_cast<const int*>(&D.org[i]);
        double X = D.Xref[3 * i + tl] + (double)dx[tl] - (double)c[tl];
        reinterpret_cast<float*>(&D.xf[i])[tl] = (float)(X - o[tl]);
    }
    if (tl == 0) {
        float4 dx = D.dX[i], v = D.V[i];
        float dd = sqrtf(dx.x * dx.x + dx.y * dx.y + dx.z * dx.z);
        float vv = sqrtf(v.x * v.x + v.y * v.y + v.z * v.z);
        if (!(dd == dd) || !(vv == vv) || isinf(dd) || isinf(vv)) bad |= ST_UNSTABLE;
        else if (dd >= D.hard_disp) bad |= ST_SKIN;
        dmax = fmaxf(dmax, dd);
        vmax = fmaxf(vmax, vv);
    }
}

// Warp reduction of the maxima and the status bits, one atomic each per warp
// (every lane of the warp calls it).
__device__ __forceinline__ void flush_maxima(const Dem& D, float dmax, float vmax, uint32_t bad) {
    const unsigned full = 0xffffffffu;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        dmax = fmaxf(dmax, __shfl_xor_sync(full, dmax, o));
        vmax = fmaxf(vmax, __shfl_xor_sync(full, vmax, o));
        bad |= __shfl_xor_sync(full, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (dmax > 0.f) {
            atomicMax(D.max_disp_bits, __float_as_uint(dmax));
            atomicMax(D.disp_layout_bits, __float_as_uint(dmax));
        }
        if (vmax > 0.f) atomicMax(D.max_vel_bits, __float_as_uint(vmax));
        if (bad) atomicOr(D.status, bad);
    }
}

__global__ void k_dem_step(Dem D, int init_only) {
    cg::cluster_group cl = cg::this_cluster();
    const int nth = gridDim.x * blockDim.x;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int team = tid / TEAM, tl = tid % TEAM, nteams = nth / TEAM;
    const int iters = (D.n + nteams - 1) / nteams;  // uniform: shuffles stay converged
    if (!init_only && tid == 0) *D.layout_fresh = 0u;  // this step's map update is done
    if (init_only) {
        for (int i = tid; i < D.n; i += nth) {
            D.dXb[i] = D.dX[i];
            D.Vhb[i] = D.V[i];
            D.Whb[i] = D.W[i];
        }
        cl.sync();
        for (int it = 0; it < iters; ++it) {
            int i = team + it * nteams;
            float3 F = make_float3(0.f, 0.f, 0.f), T = F;
            if (i < D.n) contact_forces(D, i, 0, 0.f, tl, F, T);
            team_sum(F, T);
            if (i < D.n && tl == 0) {
                D.Fc[i] = make_float4(F.x, F.y, F.z, 0.f);
                D.Tc[i] = make_float4(T.x, T.y, T.z, 0.f);
            }
        }
    } else {
        for (int it = 0; it < iters; ++it) {
            int i = team + it * nteams;
            if (i >= D.n || tl != 0) continue;
            double f[3] = {0.0, 0.0, 0.0}, t[3] = {0.0, 0.0, 0.0};
            for (int r = 0; r < NREP; ++r)
                for (int a = 0; a < 3; ++a) {
                    f[a] += D.Fh[3 * ((size_t)r * D.n + i) + a];
                    t[a] += D.Th[3 * ((size_t)r * D.n + i) + a];
                }
            D.Fa[i] = make_float4((float)(0.5 * (f[0] + D.Fh_prev[3 * i])), (float)(0.5 * (f[1] + D.Fh_prev[3 * i + 1])),
                                  (float)(0.5 * (f[2] + D.Fh_prev[3 * i + 2])), 0.f);
            D.Ta[i] = make_float4((float)(0.5 * (t[0] + D.Th_prev[3 * i])), (float)(0.5 * (t[1] + D.Th_prev[3 * i + 1])),
                                  (float)(0.5 * (t[2] + D.Th_prev[3 * i + 2])), 0.f);
            for (int a = 0; a < 3; ++a) {
                D.Fh_prev[3 * i + a] = f[a];
                D.Th_prev[3 * i + a] = t[a];
            }
        }
    }
    for (int s = 0; s < (init_only ? 0 : D.K); ++s) {
        const int b = s & 1;
        // kick + drift of the own spheres (lane 0 of each sphere's team owns
        // every per-sphere update, so no barrier is needed between substeps)
        for (int it = 0; it < iters; ++it) {
            int i = team + it * nteams;
            if (i >= D.n || tl != 0) continue;
            float4 dx = D.dX[i];
            float4 vh, wh;
            if (D.fixed[i]) {
                vh = wh = make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
                float3 v = f3(D.V[i]), w = f3(D.W[i]), dxx = f3(dx), c = f3(D.dXc[i]);
                float4 q = D.q[i];
                float3 vh3, wh3;
                kick_drift(D, f3(D.Fc[i]), f3(D.Tc[i]), f3(D.Fa[i]), f3(D.Ta[i]), D.invm[i], D.invI[i], v, w, vh3,
                           wh3, dxx, c, q);
                vh = make_float4(vh3.x, vh3.y, vh3.z, 0.f);
                wh = make_float4(wh3.x, wh3.y, wh3.z, 0.f);
                dx = make_float4(dxx.x, dxx.y, dxx.z, 0.f);
                D.dX[i] = dx;
                D.dXc[i] = make_float4(c.x, c.y, c.z, 0.f);
                D.q[i] = q;
            }
            D.dXb[b * D.n + i] = dx;
            D.Vhb[b * D.n + i] = vh;
            D.Whb[b * D.n + i] = wh;
        }
        cl.sync();
        // contact forces (a team per sphere) and the closing kick
        for (int it = 0; it < iters; ++it) {
            int i = team + it * nteams;
            bool act = i < D.n && !D.fixed[i];
            float3 F = make_float3(0.f, 0.f, 0.f), T = F;
            if (act) contact_forces(D, i, b, D.dt, tl, F, T);
            team_sum(F, T);
            if (i < D.n && tl == 0) {
                if (!act) {
                    D.V[i] = D.W[i] = make_float4(0.f, 0.f, 0.f, 0.f);
                    continue;
                }
                D.Fc[i] = make_float4(F.x, F.y, F.z, 0.f);
                D.Tc[i] = make_float4(T.x, T.y, T.z, 0.f);
                float3 v, w;
                close_kick(D, f3(D.Vhb[b * D.n + i]), f3(D.Whb[b * D.n + i]), F, T, f3(D.Fa[i]), f3(D.Ta[i]),
                           D.invm[i], D.invI[i], v, w);
                D.V[i] = make_float4(v.x, v.y, v.z, 0.f);
                D.W[i] = make_float4(w.x, w.y, w.z, 0.f);
            }
        }
    }
    // outputs of the step: lattice frame of every sphere, displacement and
    // speed maxima for the re-layout decision, NaN / skin checks
    float dmax = 0.f, vmax = 0.f;
    uint32_t bad = 0;
    for (int it = 0; it < iters; ++it) {
        int i = team + it * nteams;
        if (i >= D.n || tl != 0) continue;
        sphere_frame(D, i, dmax, vmax, bad);
    }
    flush_maxima(D, dmax, vmax, bad);
    cl.sync();
}

// The same K substeps with every sphere's state in registers of its team and
// the per-substep exchange (displacement and half-step velocities) in the
// distributed shared memory of the cluster: one cluster of up to 16 CTAs of
// DSM_THREADS threads, spc = blockDim / TEAM spheres per CTA, sphere j in CTA
// j / spc.  The first NBT neighbour entries of each team lane live in
// registers (with their tangential history) for the whole launch; further
// entries go through global memory.  Used when every sphere has a team.
constexpr int DSM_THREADS = 512;
constexpr int NBT = 3;

__global__ void __launch_bounds__(DSM_THREADS, 1) k_dem_step_dsm(Dem D) {
    extern __shared__ float4 xchg[];  // [2 substep parities][3: dX, Vh, Wh][spc]
    // Launched with a programmatic dependency on the link kernel: the
    // sphere state and neighbour entries (last written by the previous
    // step's DEM, long complete) are read before waiting for it; the
    // exchange sums it writes, and every write of this kernel, come after.
    cg::cluster_group cl = cg::this_cluster();
    const int spc = blockDim.x / TEAM;
    const int tl = threadIdx.x % TEAM, ls = threadIdx.x / TEAM;
    const int i = blockIdx.x * spc + ls;
    const bool have = i < D.n;
    const unsigned full = 0xffffffffu;
    const int lead = (threadIdx.x & 31) & ~(TEAM - 1);  // lane of the team's first thread
    const float3 zero = make_float3(0.f, 0.f, 0.f);
    float3 dx = zero, dxc = zero, v = zero, w = zero, fc = zero, tc = zero;
    float4 q = make_float4(1.f, 0.f, 0.f, 0.f);
    float im = 0.f, iI = 0.f, Ri = 1.f;
    bool fixed = true;
    int cnt = 0;
    if (have) {
        dx = f3(D.dX[i]);
        dxc = f3(D.dXc[i]);
        v = f3(D.V[i]);
        w = f3(D.W[i]);
        q = D.q[i];
        fc = f3(D.Fc[i]);
        tc = f3(D.Tc[i]);
        im = D.invm[i];
        iI = D.invI[i];
        Ri = D.R[i];
        fixed = D.fixed[i] != 0;
        cnt = D.nb_cnt[i];
    }
    // this lane's neighbour entries tl + u TEAM, u < NBT; the neighbour's CTA
    // rank and slot are packed as (rank << 16) | slot once, so the substeps
    // need no division by the spheres per CTA
    int nj[NBT];
    float4 ndr[NBT];
    float3 nh[NBT];
#pragma unroll
    for (int u = 0; u < NBT; ++u) {
        int k = tl + u * TEAM;
        nj[u] = -1;
        if (k < cnt) {
            size_t e = (size_t)i * D.nbmax + k;
            const int j = D.nb_j[e], rk = j / spc;
            nj[u] = (rk << 16) | (j - rk * spc);
            ndr[u] = D.nb_dref[e];
            nh[u] = f3(D.nb_ft[e]);
        }
    }
    pdl_wait();
    if (blockIdx.x == 0 && threadIdx.x == 0) *D.layout_fresh = 0u;  // this step's map update is done
    // hydrodynamic drive: the mean of this and the previous step's exchange
    // sums.  The FP64 replica sums are split over the team: lane tl < 3
    // sums force and torque component tl (same operations and order as one
    // lane would), then the team shares them.
    float hf = 0.f, ht = 0.f;
    if (have && tl < 3) {
        double f = 0.0, t = 0.0;
        for (int r = 0; r < NREP; ++r) {
            f += D.Fh[3 * ((size_t)r * D.n + i) + tl];
            t += D.Th[3 * ((size_t)r * D.n + i) + tl];
        }
        hf = (float)(0.5 * (f + D.Fh_prev[3 * i + tl]));
        ht = (float)(0.5 * (t + D.Th_prev[3 * i + tl]));
        D.Fh_prev[3 * i + tl] = f;
        D.Th_prev[3 * i + tl] = t;
        reinterpret_cast<float*>(&D.Fa[i])[tl] = hf;
        reinterpret_cast<float*>(&D.Ta[i])[tl] = ht;
    }
    const float3 fa = make_float3(__shfl_sync(full, hf, lead), __shfl_sync(full, hf, lead + 1),
                                  __shfl_sync(full, hf, lead + 2));
    const float3 ta = make_float3(__shfl_sync(full, ht, lead), __shfl_sync(full, ht, lead + 1),
                                  __shfl_sync(full, ht, lead + 2));
    for (int s = 0; s < D.K; ++s) {
        const int b = s & 1;
        float3 vh = zero, wh = zero;
        if (!fixed) kick_drift(D, fc, tc, fa, ta, im, iI, v, w, vh, wh, dx, dxc, q);
        if (have && tl == 0) {
            xchg[(b * 3 + 0) * spc + ls] = make_float4(dx.x, dx.y, dx.z, 0.f);
            xchg[(b * 3 + 1) * spc + ls] = make_float4(vh.x, vh.y, vh.z, 0.f);
            xchg[(b * 3 + 2) * spc + ls] = make_float4(wh.x, wh.y, wh.z, 0.f);
        }
        cl.sync();
        float3 F = zero, T = zero;
        if (have && !fixed) {
#pragma unroll
            for (int u = 0; u < NBT; ++u) {
                if (nj[u] < 0) continue;
                const int rk = nj[u] >> 16, lj = nj[u] & 0xffff;
                const float4* rx = cl.map_shared_rank(xchg, rk);
                float4 xj = rx[(b * 3 + 0) * spc + lj], vj = rx[(b * 3 + 1) * spc + lj],
                       wj = rx[(b * 3 + 2) * spc + lj];
                float4 h = make_float4(nh[u].x, nh[u].y, nh[u].z, 0.f);
                pair_contact(D, Ri, __ldg(&D.R[rk * spc + lj]), make_float3(xj.x - dx.x, xj.y - dx.y, xj.z - dx.z), ndr[u],
                             vh, wh, f3(vj), f3(wj), D.dt, h, F, T);
                nh[u] = f3(h);
            }
            for (int k = tl + NBT * TEAM; k < cnt; k += TEAM) {  // entries beyond the registers
                size_t e = (size_t)i * D.nbmax + k;
                int j = D.nb_j[e];
                int rk = j / spc, lj = j - rk * spc;
                const float4* rx = cl.map_shared_rank(xchg, rk);
                float4 h = D.nb_ft[e];
                float4 xjj = rx[(b * 3 + 0) * spc + lj];
                pair_contact(D, Ri, D.R[j], make_float3(xjj.x - dx.x, xjj.y - dx.y, xjj.z - dx.z), D.nb_dref[e], vh,
                             wh, f3(rx[(b * 3 + 1) * spc + lj]), f3(rx[(b * 3 + 2) * spc + lj]), D.dt, h, F, T);
                D.nb_ft[e] = h;
            }
        }
        team_sum(F, T);
        if (fixed) {
            v = w = zero;
        } else {
            fc = F;
            tc = T;
            close_kick(D, vh, wh, F, T, fa, ta, im, iI, v, w);
        }
    }
    cl.sync();  // no CTA leaves while another may still read its shared memory
    if (have) {
#pragma unroll
        for (int u = 0; u < NBT; ++u)
            if (nj[u] >= 0) D.nb_ft[(size_t)i * D.nbmax + tl + u * TEAM] = make_float4(nh[u].x, nh[u].y, nh[u].z, 0.f);
        if (tl == 0) {
            D.dX[i] = make_float4(dx.x, dx.y, dx.z, 0.f);
            D.dXc[i] = make_float4(dxc.x, dxc.y, dxc.z, 0.f);
            D.V[i] = make_float4(v.x, v.y, v.z, 0.f);
            D.W[i] = make_float4(w.x, w.y, w.z, 0.f);
            D.q[i] = q;
            D.Fc[i] = make_float4(fc.x, fc.y, fc.z, 0.f);
            D.Tc[i] = make_float4(tc.x, tc.y, tc.z, 0.f);
        }
    }
    float dmax = 0.f, vmax = 0.f;
    uint32_t bad = 0;
    __syncwarp();
    if (have) sphere_offset(D, i, tl, dmax, vmax, bad);
    flush_maxima(D, dmax, vmax, bad);
}

// Largest cluster (CTAs of DSM_THREADS threads) the DSM kernel can run with
// on each device, found on the first initialisation launch (outside any
// stream capture); 0 = not found (the general kernel serves).
static int g_dsm_cluster[64];
static bool g_dsm_probed[64];

static void probe_dsm(int dev) {
    if (dev < 0 || dev >= 64 || g_dsm_probed[dev]) return;
    g_dsm_probed[dev] = true;
    g_dsm_cluster[dev] = 0;
    if (cudaFuncSetAttribute(k_dem_step_dsm, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    for (int C : {16, 8}) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(C, 1, 1);
        cfg.blockDim = dim3(DSM_THREADS, 1, 1);
        cfg.dynamicSmemBytes = 6 * (DSM_THREADS / TEAM) * sizeof(float4);
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int ncl = 0;
        if (cudaOccupancyMaxActiveClusters(&ncl, k_dem_step_dsm, &cfg) == cudaSuccess && ncl > 0) {
            g_dsm_cluster[dev] = C;
            break;
        }
        cudaGetLastError();
    }
}

void launch_dem_step(const Dem& D, bool init_only, cudaStream_t s) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (init_only) probe_dsm(dev);
    long long need = (long long)TEAM * (D.n > 0 ? D.n : 1);
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int cmax = dev >= 0 && dev < 64 ? g_dsm_cluster[dev] : 0;
    if (!init_only && cmax > 0 && need <= (long long)cmax * DSM_THREADS) {
        // the smallest CTAs that fit the cluster: a CTA holds half an SM's
        // registers at 256 threads, so DEM clusters of concurrent columns
        // (batches) find room next to the lattice kernels
        int T = need <= (long long)cmax * (DSM_THREADS / 2) ? DSM_THREADS / 2 : DSM_THREADS;
        int C = 1;
        if (need > T) C = (int)((need + T - 1) / T);
        else T = (int)(((need + 31) / 32) * 32);
        cfg.gridDim = dim3(C, 1, 1);
        cfg.blockDim = dim3(T, 1, 1);
        cfg.dynamicSmemBytes = 6 * (T / TEAM) * sizeof(float4);
        attr[0].val.clusterDim.x = C;
        // programmatic dependency on the link kernel (pdl_wait first)
        attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[1].val.programmaticStreamSerializationAllowed = 1;
        cfg.numAttrs = 2;
        cudaLaunchKernelEx(&cfg, k_dem_step_dsm, D);
        return;
    }
    // general kernel: TEAM threads per sphere, up to 8 CTAs of up to 1024
    // threads, several spheres per team when needed
    int C = 1;
    int T = (int)(((need + 31) / 32) * 32);
    if (T > 256) {
        C = (int)std::min<long long>(D.cluster, (need + 255) / 256);
        T = (int)((need + C - 1) / C);
        T = ((T + 31) / 32) * 32;
        if (T > 1024) T = 1024;
    }
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(T, 1, 1);
    cfg.dynamicSmemBytes = 0;
    attr[0].val.clusterDim.x = C;
    cudaLaunchKernelEx(&cfg, k_dem_step, D, init_only ? 1 : 0);
}

// ------------------------------------------------------------ neighbour lists

__device__ __forceinline__ int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
__device__ __forceinline__ int floormod(int a, int b) { return a - floordiv(a, b) * b; }

// Cell of a position: periodic axes use the wrapped coordinate and return
// the wrap count k (X = X_wrapped + k L); the x axis clamps when not periodic.
__device__ __forceinline__ int cell_axis(double X, double lo, double h, int nc, double L, int periodic,
                                         int& k) {
    if (periodic) {
        k = (int)floor(X / L);
        double xw = X - k * L;
        int c = (int)floor(xw / h);
        return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
    }
    k = 0;
    int c = (int)floor((X - lo) / h);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

__global__ void k_cell_count(const double* X, int n, CellGrid G, int* cell_of, int* count) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int kx, ky, kz;
    int cx_ = cell_axis(X[3 * i], G.lo.x, G.h.x, G.nc.x, G.L.x, G.px, kx);
    int cy_ = cell_axis(X[3 * i + 1], 0.0, G.h.y, G.nc.y, G.L.y, 1, ky);
    int cz_ = cell_axis(X[3 * i + 2], 0.0, G.h.z, G.nc.z, G.L.z, 1, kz);
    int c = (cx_ * G.nc.y + cy_) * G.nc.z + cz_;
    cell_of[i] = c;
    atomicAdd(&count[c], 1);
}

__global__ void k_cell_fill(const int* cell_of, int n, int* fill, int* order) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int slot = atomicAdd(&fill[cell_of[i]], 1);
    order[slot] = i;
}

// Per sphere: all (j, image) within R_i + R_j + skin, sorted by (j, image),
// tangential history copied from the previous list where the key matches.
__global__ void k_nb_build(NbBuild B) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B.n) return;
    const CellGrid& G = B.G;
    double Xi[3] = {B.X[3 * i], B.X[3 * i + 1], B.X[3 * i + 2]};
    int ki[3];
    int ci[3];
    ci[0] = cell_axis(Xi[0], G.lo.x, G.h.x, G.nc.x, G.L.x, G.px, ki[0]);
    ci[1] = cell_axis(Xi[1], 0.0, G.h.y, G.nc.y, G.L.y, 1, ki[1]);
    ci[2] = cell_axis(Xi[2], 0.0, G.h.z, G.nc.z, G.L.z, 1, ki[2]);
    int nc[3] = {G.nc.x, G.nc.y, G.nc.z};
    int per[3] = {G.px, 1, 1};
    double L[3] = {G.L.x, G.L.y, G.L.z};
    size_t base = (size_t)i * B.nbmax;
    int cnt = 0;
    double Ri = B.R[i];
    for (int dx = -1; dx <= 1; ++dx) {
        int ux = ci[0] + dx;
        int wx = ux, sx = 0;
        if (per[0]) {
            wx = floormod(ux, nc[0]);
            sx = floordiv(ux, nc[0]);
        } else if (ux < 0 || ux >= nc[0]) {
            continue;
        }
        for (int dy = -1; dy <= 1; ++dy) {
            int uy = ci[1] + dy, wy = floormod(uy, nc[1]), sy = floordiv(uy, nc[1]);
            for (int dz = -1; dz <= 1; ++dz) {
                int uz = ci[2] + dz, wz = floormod(uz, nc[2]), sz = floordiv(uz, nc[2]);
                int c = (wx * nc[1] + wy) * nc[2] + wz;
                for (int a = B.start[c]; a < B.start[c + 1]; ++a) {
                    int j = B.order[a];
                    if (j == i) continue;
                    int kj[3];
                    cell_axis(B.X[3 * j], G.lo.x, G.h.x, G.nc.x, G.L.x, G.px, kj[0]);
                    cell_axis(B.X[3 * j + 1], 0.0, G.h.y, G.nc.y, G.L.y, 1, kj[1]);
                    cell_axis(B.X[3 * j + 2], 0.0, G.h.z, G.nc.z, G.L.z, 1, kj[2]);
                    int s[3] = {per[0] ? sx - kj[0] + ki[0] : 0, sy - kj[1] + ki[1], sz - kj[2] + ki[2]};
                    double d[3];
                    for (int q = 0; q < 3; ++q) d[q] = (B.X[3 * j + q] + s[q] * L[q]) - Xi[q];
                    double cut = Ri + B.R[j] + B.skin;
                    double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    if (dd >= cut * cut) continue;
                    if (cnt >= B.nbmax) {
                        atomicOr(B.status, ST_CAPACITY);
                        continue;
                    }
                    size_t e = base + cnt++;
                    B.nj[e] = j;
                    B.nsh[4 * e] = (int8_t)s[0];
                    B.nsh[4 * e + 1] = (int8_t)s[1];
                    B.nsh[4 * e + 2] = (int8_t)s[2];
                    B.nsh[4 * e + 3] = 0;
                    // the overlap is later formed from e0 = (R_i + R_j)^2 - |dref|^2,
                    // taken here in FP64 from the unrounded offset, so FP32 never
                    // cancels two ~2R numbers (nor carries dref's rounding)
                    double c2 = Ri + B.R[j];
                    double e0 = c2 * c2 - dd;
                    B.dref[e] = make_float4((float)d[0], (float)d[1], (float)d[2], (float)e0);
                }
            }
        }
    }
    // insertion sort by (j, sx, sy, sz)
    auto key = [&](size_t e) -> long long {
        return ((long long)B.nj[e] << 24) | ((long long)(B.nsh[4 * e] + 8) << 16) |
               ((long long)(B.nsh[4 * e + 1] + 8) << 8) | (long long)(B.nsh[4 * e + 2] + 8);
    };
    for (int a = 1; a < cnt; ++a) {
        size_t ea = base + a;
        long long ka = key(ea);
        int j = B.nj[ea];
        int8_t sh[4] = {B.nsh[4 * ea], B.nsh[4 * ea + 1], B.nsh[4 * ea + 2], 0};
        float4 dr = B.dref[ea];
        int b = a - 1;
        while (b >= 0 && key(base + b) > ka) {
            size_t eb = base + b, eb1 = base + b + 1;
            B.nj[eb1] = B.nj[eb];
            for (int q = 0; q < 4; ++q) B.nsh[4 * eb1 + q] = B.nsh[4 * eb + q];
            B.dref[eb1] = B.dref[eb];
            --b;
        }
        size_t e = base + b + 1;
        B.nj[e] = j;
        for (int q = 0; q < 4; ++q) B.nsh[4 * e + q] = sh[q];
        B.dref[e] = dr;
    }
    // carry the tangential history over
    int oc = B.old_cnt ? B.old_cnt[i] : 0;
    for (int a = 0; a < cnt; ++a) {
        size_t e = base + a;
        float4 h = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int b = 0; b < oc; ++b) {
            size_t o = base + b;
            if (B.old_j[o] == B.nj[e] && B.old_sh[4 * o] == B.nsh[4 * e] &&
                B.old_sh[4 * o + 1] == B.nsh[4 * e + 1] && B.old_sh[4 * o + 2] == B.nsh[4 * e + 2]) {
                h = B.old_ft[o];
                break;
            }
        }
        B.ft[e] = h;
    }
    B.cnt[i] = cnt;
}


void launch_cells(const double* X, int n, const CellGrid& G, int* cell_of, int* count, int* start,
                  int* fill, int* order, uint32_t* scan_tmp, cudaStream_t s) {
    int ncell = G.nc.x * G.nc.y * G.nc.z;
    // count[ncell] stays 0, so the exclusive scan of ncell + 1 counts also
    // leaves the total in start[ncell]; the fill cursors start as a copy
    cudaMemsetAsync(count, 0, sizeof(int) * (ncell + 1), s);
    if (n > 0) k_cell_count<<<(n + 255) / 256, 256, 0, s>>>(X, n, G, cell_of, count);
    exclusive_scan(reinterpret_cast<const uint32_t*>(count), reinterpret_cast<uint32_t*>(start), (size_t)ncell + 1,
                   scan_tmp, s);
    cudaMemcpyAsync(fill, start, sizeof(int) * ncell, cudaMemcpyDeviceToDevice, s);
    if (n > 0) k_cell_fill<<<(n + 255) / 256, 256, 0, s>>>(cell_of, n, fill, order);
}

void launch_nb_build(const NbBuild& B, cudaStream_t s) {
    if (B.n > 0) k_nb_build<<<(B.n + 127) / 128, 128, 0, s>>>(B);
}

// Spheres whose surface may reach a band node before the next re-layout
// (|y - Xref| < R + skin, all images), ascending, at most 4, and the node's
// slack: its distance to the nearest candidate surface.  The owner of the
// node is a function of the candidates' inside tests (and, inside two or
// more spheres, of their distance ratios), so it cannot change while every
// sphere stays closer than the slack to its layout position; a node inside
// two or more candidates, or a boundary-plane node, is flagged 0 (always
// re-tested) or never changes (planes stay fluid) respectively.
__global__ void k_band_cand(BandCand B) {
    uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= B.n) return;
    const CellGrid& G = B.G;
    int x, y, z;
    unpack_coord(B.coord[k], x, y, z);
    double P[3] = {(double)x, (double)y, (double)z};
    int kk[3], ci[3];
    ci[0] = cell_axis(P[0], G.lo.x, G.h.x, G.nc.x, G.L.x, G.px, kk[0]);
    ci[1] = cell_axis(P[1], 0.0, G.h.y, G.nc.y, G.L.y, 1, kk[1]);
    ci[2] = cell_axis(P[2], 0.0, G.h.z, G.nc.z, G.L.z, 1, kk[2]);
    int nc[3] = {G.nc.x, G.nc.y, G.nc.z};
    double L[3] = {G.L.x, G.L.y, G.L.z};
    const double iL[3] = {1.0 / G.L.x, 1.0 / G.L.y, 1.0 / G.L.z};  // once per node, not per candidate
    int per[3] = {G.px, 1, 1};
    int c4[4] = {-1, -1, -1, -1};
    int nfound = 0, ninside = 0;
    double slack = 1e30;
    for (int dx = -1; dx <= 1; ++dx) {
        int ux = ci[0] + dx, wx = ux;
        if (per[0]) wx = floormod(ux, nc[0]);
        else if (ux < 0 || ux >= nc[0]) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            int wy = floormod(ci[1] + dy, nc[1]);
            for (int dz = -1; dz <= 1; ++dz) {
                int wz = floormod(ci[2] + dz, nc[2]);
                int c = (wx * nc[1] + wy) * nc[2] + wz;
                for (int a = B.start[c]; a < B.start[c + 1]; ++a) {
                    int p = B.order[a];
                    bool dup = false;
                    for (int q = 0; q < nfound; ++q) dup |= c4[q] == p;
                    if (dup) continue;
                    double d2 = 0;
                    for (int q = 0; q < 3; ++q) {
                        double d = P[q] - B.X[3 * p + q];
                        if (per[q]) d -= L[q] * floor(d * iL[q] + 0.5);
                        d2 += d * d;
                    }
                    double r = B.R[p] + B.skin;
                    if (d2 >= r * r) continue;
                    slack = fmin(slack, fabs(sqrt(d2) - B.R[p]));
                    ninside += d2 < B.R[p] * B.R[p];
                    if (nfound >= 4) {
                        atomicOr(B.status, ST_CAPACITY);
                        continue;
                    }
                    // insert sorted
                    int q = nfound++;
                    while (q > 0 && c4[q - 1] > p) {
                        c4[q] = c4[q - 1];
                        --q;
                    }
                    c4[q] = p;
                }
            }
        }
    }
    B.cand[k] = make_int4(c4[0], c4[1], c4[2], c4[3]);
    if (ninside >= 2) slack = 0.0;
    if (!G.px && (x == 0 || x == B.nx - 1)) slack = 1e30;  // inlet/outlet planes stay fluid
    B.slack[k] = (float)slack;
    if (B.band_dense) B.band_dense[((size_t)x * B.ny + y) * B.nz + z] = nfound >= 2 ? 2 : 1;
}

void launch_band_cand(const BandCand& B, cudaStream_t s) {
    if (B.n > 0) k_band_cand<<<(B.n + 255) / 256, 256, 0, s>>>(B);
}

// Band list ordered by slack (bucket sort, order inside a bucket arbitrary):
// the nodes a step has to re-test -- slack up to the displacement since the
// layout -- then form a prefix of the list and fill whole warps, and the
// warps past it leave after one coalesced load.
constexpr int SLACK_BUCKETS = 1024;
static_assert(SLACK_HIST == SLACK_BUCKETS + 1, "bucket counts and the total");
__device__ __forceinline__ int slack_bucket(float slack, float top) {
    float b = slack * (float)SLACK_BUCKETS / top;
    return b < (float)(SLACK_BUCKETS - 1) ? (int)b : SLACK_BUCKETS - 1;
}
__global__ void k_slack_hist(const float* slack, uint32_t n, float top, uint32_t* hist) {
    uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) atomicAdd(&hist[slack_bucket(slack[k], top)], 1u);
}
__global__ void k_slack_scatter(const uint32_t* coord, const int4* cand, const float* slack, uint32_t n, float top,
                                uint32_t* next, uint32_t* coord2, int4* cand2, float* slack2) {
    uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    uint32_t pos = atomicAdd(&next[slack_bucket(slack[k], top)], 1u);
    coord2[pos] = coord[k];
    cand2[pos] = cand[k];
    slack2[pos] = slack[k];
}
void launch_band_sort(const uint32_t* coord, const int4* cand, const float* slack, uint32_t n, double skin,
                      uint32_t* hist, uint32_t* scan_tmp, uint32_t* coord2, int4* cand2, float* slack2,
                      cudaStream_t s) {
    if (n == 0) return;
    const float top = (float)(2.0 * skin);  // band nodes lie within skin of a surface
    cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (SLACK_BUCKETS + 1), s);
    k_slack_hist<<<(n + 255) / 256, 256, 0, s>>>(slack, n, top, hist);
    exclusive_scan(hist, hist, SLACK_BUCKETS + 1, scan_tmp, s);
    k_slack_scatter<<<(n + 255) / 256, 256, 0, s>>>(coord, cand, slack, n, top, hist, coord2, cand2, slack2);
}

__global__ void k_rebase(double* Xref, float4* dX, float4* dXc, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 d = dX[i], c = dXc[i];
    Xref[3 * i] += (double)d.x - (double)c.x;
    Xref[3 * i + 1] += (double)d.y - (double)c.y;
    Xref[3 * i + 2] += (double)d.z - (double)c.z;
    dX[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    dXc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

void launch_rebase(double* Xref, float4* dX, float4* dXc, int n, cudaStream_t s) {
    if (n > 0) k_rebase<<<(n + 255) / 256, 256, 0, s>>>(Xref, dX, dXc, n);
}

}  // namespace lbmdem
