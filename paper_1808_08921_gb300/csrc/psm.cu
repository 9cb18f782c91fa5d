// psm.cu -- a smooth surrogate of the fluid-solid coupling, for the gradient
// of the probe-plane pressure misfit with respect to the sphere positions of
// a fixed packing.  It lies outside the paper's chosen method: with the
// binary solid map of the momentum-exchange coupling (Section 2.3, Eqs.
// 14-15) the misfit is piecewise constant in the centres, so the gradient is
// taken of a surrogate from the family the paper names as the alternative
// (Section 1: Noble and Torczynski's collision weighted by the solid volume
// fraction of each cell).
//
// Model (dense lattice, every node carries populations, deviations
// g = f - w rho_f, FP32 arithmetic):
//   * solid fraction eps(x) = 1 - prod_p (1 - S(R_p - |x - X_p| + 1/2)), S the
//     cubic smoothstep (0 below 0, 3 s^2 - 2 s^3 on [0, 1], 1 above), the
//     distance to the nearest periodic image; the x ends of a non-periodic
//     lattice stay fluid;
//   * collision  g*_i = g_i - a (g_i - g^eq_i) + B Om_i,  a = (1 - B)/tau,
//     B = eps (tau - 1/2) / ((1 - eps) + (tau - 1/2)),
//     Om_i = g_opp(i) - g_i + w_i drho - g^eq_opp(i)  (the bounce-back of the
//     non-equilibrium part towards a resting solid);
//   * streaming of every population to x + c_i; a population leaving the x
//     range comes back reversed (resting wall); then the pressure inlet
//     (Zou-He, Eq. 25) and the outlet, as in the coupled step;
//   * probe: c_s^2 times the mean density over every node of plane probe_x.
// Reverse mode, for L = sum_k l_k(g_k) and the adjoint lam_k = dL/dg_k:
//   mu = S^T B^T lam_{k+1} (the adjoint of the post-collision state:
//   mu_i(x) = lam_i(x + c_i), or lam_opp(i)(x) where the population left the
//   lattice), then
//   lam_k = (1 - a - B) mu + B mu_opp + B (w . mu) 1 + A(nu) + Bv(nu) . c + dl_k/dg_k,
//   nu_i = a mu_i - B mu_opp(i), A and Bv the contractions of nu with
//   dg^eq/d(drho) and dg^eq/dJ;
//   dL/dtau += mu . dg*/dtau, G(x) += mu . dg*/deps at every node, and at the
//   end dL/dX_p = sum_x G(x) deps(x)/dX_p.
#include "common.cuh"
#include "kernels.cuh"

namespace lbmdem {

__device__ __forceinline__ size_t dense(const PsmArgs& A, int x, int y, int z) {
    return ((size_t)x * A.ny + y) * A.nz + z;
}

// node of this thread in the 3-D launch of psm_grid: z along the block's
// threads, y and x from the block indices (no integer division); false past
// the end of a z line
__device__ __forceinline__ bool grid_node(const PsmArgs& A, int& x, int& y, int& z, size_t& k) {
    z = blockIdx.x * blockDim.x + threadIdx.x;
    y = blockIdx.y;
    x = blockIdx.z;
    k = dense(A, x, y, z);
    return z < A.nz;
}

__device__ __forceinline__ double smooth_step(double v) {
    if (v <= 0.0) return 0.0;
    if (v >= 1.0) return 1.0;
    return v * v * (3.0 - 2.0 * v);
}

// node offset from a centre along one axis, nearest periodic image
__device__ __forceinline__ double image(double d, double L, bool periodic) {
    return periodic ? d - L * floor(d / L + 0.5) : d;
}

__global__ void k_psm_eps(PsmArgs A, const double* X, const double* R, int n, float* eps) {
    int x, y, z;
    size_t k;
    if (!grid_node(A, x, y, z, k)) return;
    if (!A.px && (x == 0 || x == A.nx - 1)) {
        eps[k] = 0.f;
        return;
    }
    double keep = 1.0;
    for (int p = 0; p < n; ++p) {
        const double rx = image(x - X[3 * p], A.nx, A.px), ry = image(y - X[3 * p + 1], A.ny, true),
                     rz = image(z - X[3 * p + 2], A.nz, true);
        const double d2 = rx * rx + ry * ry + rz * rz, reach = R[p] + 0.5;
        if (d2 >= reach * reach) continue;
        keep *= 1.0 - smooth_step(R[p] - sqrt(d2) + 0.5);
    }
    eps[k] = (float)(1.0 - keep);
}

// collision weights of a node: B, a = (1 - B)/tau
__device__ __forceinline__ void psm_weights(float e, float tau, float& B, float& a) {
    const float sh = tau - 0.5f;
    B = e * sh / ((1.0f - e) + sh);
    a = (1.0f - B) / tau;
}

// moments and equilibrium deviations of a node
__device__ __forceinline__ void psm_eq(const float g[Q], float rho_f, float& drho, float& ux, float& uy, float& uz,
                                       float geq[Q]) {
    drho = 0.f;
    float jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int m = 0; m < Q; ++m) {
        drho += g[m];
        jx += cx(m) * g[m];
        jy += cy(m) * g[m];
        jz += cz(m) * g[m];
    }
    const float rho = rho_f + drho, ir = 1.0f / rho;
    ux = jx * ir;
    uy = jy * ir;
    uz = jz * ir;
    const float uu15 = 1.5f * (ux * ux + uy * uy + uz * uz);
#pragma unroll
    for (int m = 0; m < Q; ++m) {
        const float cu = cx(m) * ux + cy(m) * uy + cz(m) * uz;
        geq[m] = wt(m) * (drho + rho * (3.0f * cu + 4.5f * cu * cu - uu15));
    }
}

__global__ void __launch_bounds__(256) k_psm_step(PsmArgs A, const float* gin, float* gout, const float* eps) {
    int x, y, z;
    size_t k;
    if (!grid_node(A, x, y, z, k)) return;
    float g[Q], geq[Q];
#pragma unroll
    for (int m = 0; m < Q; ++m) g[m] = gin[(size_t)m * A.N + k];
    float drho, ux, uy, uz;
    psm_eq(g, A.rho_f, drho, ux, uy, uz, geq);
    float B, a;
    psm_weights(eps[k], A.tau, B, a);
    const int ym = y == 0 ? A.ny - 1 : y - 1, yp = y == A.ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? A.nz - 1 : z - 1, zp = z == A.nz - 1 ? 0 : z + 1;
#pragma unroll
    for (int m = 0; m < Q; ++m) {
        const float gs = g[m] - a * (g[m] - geq[m]) + B * (g[opp(m)] - g[m] + wt(m) * drho - geq[opp(m)]);
        int xs = x + cx(m);
        if (A.px) {
            xs = xs < 0 ? A.nx - 1 : (xs >= A.nx ? 0 : xs);
        } else if (xs < 0 || xs >= A.nx) {
            gout[(size_t)opp(m) * A.N + k] = gs;  // resting wall at the x ends
            continue;
        }
        const int ys = cy(m) > 0 ? yp : (cy(m) < 0 ? ym : y), zs = cz(m) > 0 ? zp : (cz(m) < 0 ? zm : z);
        gout[(size_t)m * A.N + dense(A, xs, ys, zs)] = gs;
    }
}

// the pressure inlet and the outlet on the state t + 1 (one thread per line)
__global__ void k_psm_boundary(PsmArgs A, float* g, Source src, unsigned long long t1) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= A.ny * A.nz) return;
    const int y = k / A.nz, z = k - y * A.nz;
    if (A.inlet == 0) {
        const size_t i = dense(A, 0, y, z);
        float f[Q];
#pragma unroll
        for (int m = 0; m < Q; ++m) f[m] = g[(size_t)m * A.N + i];
        pressure_face(f, (float)source_drho(src, t1), 0);
#pragma unroll
        for (int m = 0; m < Q; ++m)
            if (cx(m) > 0) g[(size_t)m * A.N + i] = f[m];
    }
    const size_t o = dense(A, A.nx - 1, y, z);
    if (A.outlet == 0) {
        const size_t u = dense(A, A.nx - 2, y, z);
#pragma unroll
        for (int m = 0; m < Q; ++m)
            if (cx(m) < 0) g[(size_t)m * A.N + o] = g[(size_t)m * A.N + u];
    } else if (A.outlet == 1) {
        float f[Q];
#pragma unroll
        for (int m = 0; m < Q; ++m) f[m] = g[(size_t)m * A.N + o];
        pressure_face(f, 0.f, 1);
#pragma unroll
        for (int m = 0; m < Q; ++m)
            if (cx(m) < 0) g[(size_t)m * A.N + o] = f[m];
    }
}

// sum of the density deviations over plane probe_x (FP64 atomics per warp)
__global__ void k_psm_probe(PsmArgs A, const float* g, double* out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (k < A.ny * A.nz) {
        const size_t i = dense(A, A.probe_x, k / A.nz, k % A.nz);
        float d = 0.f;
#pragma unroll
        for (int m = 0; m < Q; ++m) d += g[(size_t)m * A.N + i];
        s = d;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(out, s);
}

// B^T in place on the adjoint of the state t + 1 (the transposed Zou-He face
// and outlet) and the amplitude derivative d rho_in / d rho' = shape(t + 1)
__global__ void k_psm_adj_boundary(PsmArgs A, float* a, double shape, double* d_amp) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    double da = 0.0;
    if (k < A.ny * A.nz) {
        const int y = k / A.nz, z = k - y * A.nz;
        const size_t P = A.N;
        if (A.inlet == 0) {
            const size_t i = dense(A, 0, y, z);
            const float a0 = a[0 * P + i], a6 = a[6 * P + i], a7 = a[7 * P + i], a8 = a[8 * P + i],
                        a9 = a[9 * P + i];
            const float ar = a0 * (1.f / 3.f) + (a6 + a7 + a8 + a9) * (1.f / 6.f);
            const float ay = 0.5f * (a7 - a6), az = 0.5f * (a9 - a8);
            a[1 * P + i] += a0 - 2.f * ar;
            a[11 * P + i] += a6 - 2.f * ar;
            a[10 * P + i] += a7 - 2.f * ar;
            a[13 * P + i] += a8 - 2.f * ar;
            a[12 * P + i] += a9 - 2.f * ar;
            a[18 * P + i] += -ar;
            a[2 * P + i] += -ar + ay;
            a[3 * P + i] += -ar - ay;
            a[4 * P + i] += -ar + az;
            a[5 * P + i] += -ar - az;
            a[14 * P + i] += -ar + ay + az;
            a[15 * P + i] += -ar + ay - az;
            a[16 * P + i] += -ar - ay + az;
            a[17 * P + i] += -ar - ay - az;
            a[0 * P + i] = a[6 * P + i] = a[7 * P + i] = a[8 * P + i] = a[9 * P + i] = 0.f;
            da = (double)ar * shape;
        }
        const size_t o = dense(A, A.nx - 1, y, z);
        if (A.outlet == 0) {
            const size_t u = dense(A, A.nx - 2, y, z);
            const int um[5] = {1, 10, 11, 12, 13};
            for (int q = 0; q < 5; ++q) {
                a[um[q] * P + u] += a[um[q] * P + o];
                a[um[q] * P + o] = 0.f;
            }
        } else if (A.outlet == 1) {
            const float a1 = a[1 * P + o], a11 = a[11 * P + o], a10 = a[10 * P + o], a13 = a[13 * P + o],
                        a12 = a[12 * P + o];
            const float ar = -(a1 * (1.f / 3.f) + (a11 + a10 + a13 + a12) * (1.f / 6.f));
            const float ay = 0.5f * (a11 - a10), az = 0.5f * (a13 - a12);
            a[0 * P + o] += a1 + 2.f * ar;
            a[6 * P + o] += a11 + 2.f * ar;
            a[7 * P + o] += a10 + 2.f * ar;
            a[8 * P + o] += a13 + 2.f * ar;
            a[9 * P + o] += a12 + 2.f * ar;
            a[18 * P + o] += ar;
            a[2 * P + o] += ar + ay;
            a[3 * P + o] += ar - ay;
            a[4 * P + o] += ar + az;
            a[5 * P + o] += ar - az;
            a[14 * P + o] += ar + ay + az;
            a[15 * P + o] += ar + ay - az;
            a[16 * P + o] += ar - ay + az;
            a[17 * P + o] += ar - ay - az;
            a[1 * P + o] = a[11 * P + o] = a[10 * P + o] = a[13 * P + o] = a[12 * P + o] = 0.f;
        }
    }
#pragma unroll
    for (int s = 16; s; s >>= 1) da += __shfl_xor_sync(0xffffffffu, da, s);
    if ((threadIdx.x & 31) == 0 && da != 0.0) atomicAdd(d_amp, da);
}

// lam_k = J^T mu + dl_k / dg_k at every node, with the tau and eps derivatives
__global__ void __launch_bounds__(256) k_psm_adj_step(PsmArgs A, const float* lin, const float* gt, float* lout,
                                                      const float* eps, float dl, double* d_tau, double* G) {
    int x, y, z;
    size_t k;
    double dt = 0.0;
    if (grid_node(A, x, y, z, k)) {
        const int ym = y == 0 ? A.ny - 1 : y - 1, yp = y == A.ny - 1 ? 0 : y + 1;
        const int zm = z == 0 ? A.nz - 1 : z - 1, zp = z == A.nz - 1 ? 0 : z + 1;
        float mu[Q];
#pragma unroll
        for (int m = 0; m < Q; ++m) {  // S^T: pull the adjoint back along c_m
            int xs = x + cx(m);
            bool out = false;
            if (A.px) xs = xs < 0 ? A.nx - 1 : (xs >= A.nx ? 0 : xs);
            else out = xs < 0 || xs >= A.nx;
            const int ys = cy(m) > 0 ? yp : (cy(m) < 0 ? ym : y), zs = cz(m) > 0 ? zp : (cz(m) < 0 ? zm : z);
            mu[m] = out ? lin[(size_t)opp(m) * A.N + k] : lin[(size_t)m * A.N + dense(A, xs, ys, zs)];
        }
        float g[Q], geq[Q];
#pragma unroll
        for (int m = 0; m < Q; ++m) g[m] = gt[(size_t)m * A.N + k];
        float drho, ux, uy, uz;
        psm_eq(g, A.rho_f, drho, ux, uy, uz, geq);
        const float e = eps[k], tau = A.tau, sh = tau - 0.5f, den = (1.0f - e) + sh;
        float B, a;
        psm_weights(e, tau, B, a);
        const float dB_dtau = e * (1.0f - e) / (den * den), dB_de = sh * (1.0f + sh) / (den * den);
        const float da_dtau = -dB_dtau / tau - (1.0f - B) / (tau * tau);
        const float uu = ux * ux + uy * uy + uz * uz;
        float Aa = 0.f, Bx = 0.f, By = 0.f, Bz = 0.f, wmu = 0.f, st = 0.f, se = 0.f;
#pragma unroll
        for (int m = 0; m < Q; ++m) {
            const float om = g[opp(m)] - g[m] + wt(m) * drho - geq[opp(m)];
            st += mu[m] * (-da_dtau * (g[m] - geq[m]) + dB_dtau * om);
            se += mu[m] * (dB_de * ((g[m] - geq[m]) / tau + om));
            wmu += wt(m) * mu[m];
            const float nu = a * mu[m] - B * mu[opp(m)];
            const float cu = cx(m) * ux + cy(m) * uy + cz(m) * uz;
            const float wn = wt(m) * nu;
            Aa += wn * (1.0f - 4.5f * cu * cu + 1.5f * uu);
            const float kk = 3.0f + 9.0f * cu;
            Bx += wn * (kk * cx(m) - 3.0f * ux);
            By += wn * (kk * cy(m) - 3.0f * uy);
            Bz += wn * (kk * cz(m) - 3.0f * uz);
        }
        const float add = x == A.probe_x ? dl : 0.f;
#pragma unroll
        for (int m = 0; m < Q; ++m)
            lout[(size_t)m * A.N + k] = (1.0f - a - B) * mu[m] + B * mu[opp(m)] + B * wmu + Aa + Bx * cx(m) +
                                        By * cy(m) + Bz * cz(m) + add;
        G[k] += (double)se;
        dt = (double)st;
    }
    block_sum_to(dt, d_tau + (blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)) % GRAD_COPIES);
}

// dL/dX_p = sum_x G(x) deps(x)/dX_p over the shell where sphere p's
// smoothstep varies (one block per sphere); deps/deps_p = (1 - eps)/(1 - eps_p)
// is the product over the other spheres, deps_p/dX_p = S'(s) (x - X_p)/d
__global__ void k_psm_grad_x(PsmArgs A, const double* G, const float* eps, const double* X, const double* R,
                             double* dX) {
    const int p = blockIdx.x;
    const double X0 = X[3 * p], X1 = X[3 * p + 1], X2 = X[3 * p + 2], Rp = R[p];
    const double reach = Rp + 0.5;
    const int x0 = (int)floor(X0 - reach), x1 = (int)ceil(X0 + reach);
    const int y0 = (int)floor(X1 - reach), y1 = (int)ceil(X1 + reach);
    const int z0 = (int)floor(X2 - reach), z1 = (int)ceil(X2 + reach);
    const int ey = y1 - y0 + 1, ez = z1 - z0 + 1;
    const long long vol = (long long)(x1 - x0 + 1) * ey * ez;
    double s[3] = {0.0, 0.0, 0.0};
    for (long long t = threadIdx.x; t < vol; t += blockDim.x) {
        const int zi = z0 + (int)(t % ez), yi = y0 + (int)((t / ez) % ey), xi = x0 + (int)(t / ((long long)ey * ez));
        int x = xi;
        if (A.px) x = ((x % A.nx) + A.nx) % A.nx;
        else if (x <= 0 || x >= A.nx - 1) continue;  // fluid x ends
        const int y = ((yi % A.ny) + A.ny) % A.ny, z = ((zi % A.nz) + A.nz) % A.nz;
        const double rx = (double)xi - X0, ry = (double)yi - X1, rz = (double)zi - X2;
        const double d = sqrt(rx * rx + ry * ry + rz * rz);
        const double v = Rp - d + 0.5;
        if (v <= 0.0 || v >= 1.0 || d == 0.0) continue;
        const double ep = smooth_step(v), dS = 6.0 * v * (1.0 - v);
        const size_t k = dense(A, x, y, z);
        const double f = G[k] * (1.0 - (double)eps[k]) / (1.0 - ep) * dS / d;
        s[0] += f * rx;
        s[1] += f * ry;
        s[2] += f * rz;
    }
    __shared__ double red[3][32];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int o = 16; o; o >>= 1) s[a] += __shfl_xor_sync(0xffffffffu, s[a], o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
        for (int a = 0; a < 3; ++a) red[a][wid] = s[a];
    __syncthreads();
    if (threadIdx.x < 3) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[threadIdx.x][w];
        dX[3 * p + threadIdx.x] = tot;
    }
}

// one thread per node: z lines in blocks of up to 256 threads, one block row
// per (y, x)
static void psm_grid(const PsmArgs& A, dim3& grid, dim3& block) {
    const int tz = A.nz >= 256 ? 256 : ((A.nz + 31) / 32) * 32;
    block = dim3(tz, 1, 1);
    grid = dim3((A.nz + tz - 1) / tz, A.ny, A.nx);
}

void launch_psm_eps(const PsmArgs& A, const double* X, const double* R, int n, float* eps, cudaStream_t s) {
    dim3 g, b;
    psm_grid(A, g, b);
    k_psm_eps<<<g, b, 0, s>>>(A, X, R, n, eps);
}
void launch_psm_step(const PsmArgs& A, const float* gin, float* gout, const float* eps, cudaStream_t s) {
    dim3 g, b;
    psm_grid(A, g, b);
    k_psm_step<<<g, b, 0, s>>>(A, gin, gout, eps);
}
void launch_psm_boundary(const PsmArgs& A, float* g, const Source& src, unsigned long long t1, cudaStream_t s) {
    if (A.px) return;
    const int n = A.ny * A.nz;
    k_psm_boundary<<<(n + 127) / 128, 128, 0, s>>>(A, g, src, t1);
}
void launch_psm_probe(const PsmArgs& A, const float* g, double* out, cudaStream_t s) {
    const int n = A.ny * A.nz;
    k_psm_probe<<<(n + 127) / 128, 128, 0, s>>>(A, g, out);
}
void launch_psm_adj_boundary(const PsmArgs& A, float* lam, double shape, double* d_amp, cudaStream_t s) {
    if (A.px) return;
    const int n = A.ny * A.nz;
    k_psm_adj_boundary<<<(n + 127) / 128, 128, 0, s>>>(A, lam, shape, d_amp);
}
void launch_psm_adj_step(const PsmArgs& A, const float* lin, const float* gt, float* lout, const float* eps, float dl,
                         double* d_tau, double* G, cudaStream_t s) {
    dim3 g, b;
    psm_grid(A, g, b);
    k_psm_adj_step<<<g, b, 0, s>>>(A, lin, gt, lout, eps, dl, d_tau, G);
}
void launch_psm_grad_x(const PsmArgs& A, const double* G, const float* eps, const double* X, const double* R, int n,
                       double* dX, cudaStream_t s) {
    if (n > 0) k_psm_grad_x<<<n, 256, 0, s>>>(A, G, eps, X, R, dX);
}

}  // namespace lbmdem
