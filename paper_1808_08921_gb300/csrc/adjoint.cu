// adjoint.cu -- reverse-mode (adjoint) kernels of the lattice step for a
// fixed packing, for the gradient of a probe-plane pressure misfit with
// respect to the relaxation time tau and the source amplitude rho'.
//
// With every sphere fixed the coupled step t -> t+1 acts on the natural
// populations n_t (the state entering step t) as
//     n_{t+1} = B_{t+1}( S( C(n_t) ) )
// C: BGK collision at every fluid node (Eqs. 4, 6, 7); S: streaming with
// half-way bounce-back at resting walls, n(x, i) <- n*(x - c_i, i) when
// x - c_i is fluid, else n*(x, opp(i)) (Eqs. 5, 14 with V_b = 0; populations
// from outside the x range reflect the same way); B: the pressure inlet
// (Zou-He, Section 2.4, density rho_f + rho' shape(t+1)) and the outlet.
// For L = sum_t l_t(n_t) the adjoint a_t = dL/dn_t obeys
//     a_t = dl_t/dn_t + J_C(n_t)^T S^T B_{t+1}^T a_{t+1},   a_T = 0,
// and dL/domega = -sum_t (S^T B^T a_{t+1}) . (n_t - n^eq(n_t)) with
// omega = 1/tau, dL/drho' = sum_t (dB_{t+1}/drho_in)^T a_{t+1} shape(t+1).
//   * S^T: s(y, j) = b(y + c_j, j) when y + c_j is fluid, else b(y, opp(j));
//   * J_C^T: n* = (1 - omega) n + omega n^eq(rho, J) with rho = sum n,
//     J = sum c n, so (J_C^T s)_j = (1 - omega) s_j + omega (A + B . c_j),
//     A = sum_i s_i dn^eq_i/drho, B = sum_i s_i dn^eq_i/dJ;
//   * B^T at an inlet node moves the adjoint of the five unknowns onto the
//     knowns through the transposed Zou-He formulas; at a zero-gradient
//     outlet it adds the unknowns' adjoint to the upstream node.
// Populations are deviations g = n - w rho_f throughout (the derivatives are
// the same).  The forward states come from the product path itself: the
// snapshot kernel reads the natural populations out of the AA layout.
#include "common.cuh"
#include "kernels.cuh"

namespace lbmdem {

// natural populations of every fluid stored node, [19][nSpad] FP32
template <int ST>
__global__ void k_adj_snapshot(Lat L, bool after_even, float* nat) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L.nS || !fluid_bit(L, i)) return;
    int x, y, z;
    unpack_coord(L.coord[i], x, y, z);
#pragma unroll
    for (int m = 0; m < Q; ++m)
        nat[(size_t)m * L.nSpad + i] = to_f<ST>(*pop_loc<ST>(L, after_even, x, y, z, i, m), L.fsi);
}

void launch_adj_snapshot(const Lat& L, bool after_even, float* nat, cudaStream_t s) {
    unsigned blocks = (L.nS + 255) / 256;
    if (!blocks) return;
    if (L.st == 0) k_adj_snapshot<0><<<blocks, 256, 0, s>>>(L, after_even, nat);
    else if (L.st == 1) k_adj_snapshot<1><<<blocks, 256, 0, s>>>(L, after_even, nat);
    else k_adj_snapshot<2><<<blocks, 256, 0, s>>>(L, after_even, nat);
}

// neighbour table: nbr[m][i] = compact index of x_i + c_m if fluid, else NONE
__global__ void k_adj_nbr(Lat L, uint32_t* nbr) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L.nS) return;
    int x, y, z;
    unpack_coord(L.coord[i], x, y, z);
#pragma unroll
    for (int m = 0; m < Q - 1; ++m) nbr[(size_t)m * L.nSpad + i] = fluid_index(L, x, y, z, cx(m), cy(m), cz(m));
}

void launch_adj_nbr(const Lat& L, uint32_t* nbr, cudaStream_t s) {
    if (L.nS) k_adj_nbr<<<(L.nS + 255) / 256, 256, 0, s>>>(L, nbr);
}

// B^T in place on the adjoint of n_{t+1}: one thread per boundary node pair
// (inlet node of a (y, z) line, outlet node and its upstream node).
__global__ void k_adj_boundary(AdjArgs A, double shape, double* d_amp) {
    const Lat& L = A.L;
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    double da = 0.0;
    if (k < L.ny * L.nz) {
        int y = k / L.nz, z = k - (k / L.nz) * L.nz;
        float* a = A.adj;
        size_t P = L.nSpad;
        bool fl;
        if (A.inlet == 0) {
            uint32_t i = stored_index(L, 0, y, z, fl);
            if (fl && i != NONE) {
                float a0 = a[0 * P + i], a6 = a[6 * P + i], a7 = a[7 * P + i], a8 = a[8 * P + i],
                      a9 = a[9 * P + i];
                // transposed x-normal Zou-He face (the forward formulas are
                // linear in the knowns and in the boundary density)
                float ar = a0 * (1.f / 3.f) + (a6 + a7 + a8 + a9) * (1.f / 6.f);
                float ay = 0.5f * (a7 - a6), az = 0.5f * (a9 - a8);
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
        }
        if (A.outlet == 0 || A.outlet == 1) {
            uint32_t o = stored_index(L, L.nx - 1, y, z, fl);
            if (fl && o != NONE) {
                if (A.outlet == 0) {  // zero gradient: unknowns copied from upstream
                    bool ufl;
                    uint32_t u = stored_index(L, L.nx - 2, y, z, ufl);
                    if (ufl && u != NONE) {
                        const int um[5] = {1, 10, 11, 12, 13};
                        for (int q = 0; q < 5; ++q) {
                            a[um[q] * P + u] += a[um[q] * P + o];
                            a[um[q] * P + o] = 0.f;
                        }
                    }
                } else {  // pressure face at rho_f: the mirrored transpose
                    float a1 = a[1 * P + o], a11 = a[11 * P + o], a10 = a[10 * P + o], a13 = a[13 * P + o],
                          a12 = a[12 * P + o];
                    // forward: rux = rest + 2 (g0 + g6 + g7 + g8 + g9) - drho_b;
                    // g1 = g0 - rux/3, g11 = g6 - rux/6 + Ny, g10 = g7 - rux/6 - Ny,
                    // g13 = g8 - rux/6 + Nz, g12 = g9 - rux/6 - Nz
                    float ar = -(a1 * (1.f / 3.f) + (a11 + a10 + a13 + a12) * (1.f / 6.f));
                    float ay = 0.5f * (a11 - a10), az = 0.5f * (a13 - a12);
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
        }
    }
    // block sum of the amplitude derivative, one FP64 atomic per warp
    const unsigned full = 0xffffffffu;
#pragma unroll
    for (int o = 16; o; o >>= 1) da += __shfl_xor_sync(full, da, o);
    if ((threadIdx.x & 31) == 0 && da != 0.0) atomicAdd(d_amp, da);
}

void launch_adj_boundary(const AdjArgs& A, double shape, double* d_amp, cudaStream_t s) {
    int n = A.L.ny * A.L.nz;
    if (A.L.px) return;
    k_adj_boundary<<<(n + 127) / 128, 128, 0, s>>>(A, shape, d_amp);
}

// a_t = J_C(n_t)^T S^T b + dl_t/dn_t, and the omega derivative
__global__ void __launch_bounds__(256) k_adj_step(AdjArgs A, const float* nat, float* out, float dl,
                                                  double* d_omega) {
    const Lat& L = A.L;
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    double dw = 0.0;
    if (i < L.nS && fluid_bit(L, i)) {
        const size_t P = L.nSpad;
        float s[Q];
#pragma unroll
        for (int j = 0; j < Q - 1; ++j) {
            uint32_t d = A.nbr[(size_t)j * P + i];
            s[j] = d != NONE ? A.adj[(size_t)j * P + d] : A.adj[(size_t)opp(j) * P + i];
        }
        s[18] = A.adj[(size_t)18 * P + i];
        float g[Q];
        float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
        for (int m = 0; m < Q; ++m) {
            g[m] = nat[(size_t)m * P + i];
            drho += g[m];
            jx += cx(m) * g[m];
            jy += cy(m) * g[m];
            jz += cz(m) * g[m];
        }
        const float rho = L.rho_f + drho, ir = 1.0f / rho;
        const float ux = jx * ir, uy = jy * ir, uz = jz * ir;
        const float uu = ux * ux + uy * uy + uz * uz;
        const float om = L.tau_inv;
        float Aa = 0.f, Bx = 0.f, By = 0.f, Bz = 0.f, sw = 0.f;
#pragma unroll
        for (int m = 0; m < Q; ++m) {
            float cu = cx(m) * ux + cy(m) * uy + cz(m) * uz;
            float geq = wt(m) * (drho + rho * (3.0f * cu + 4.5f * cu * cu - 1.5f * uu));
            sw += s[m] * (g[m] - geq);
            float ws = wt(m) * s[m];
            Aa += ws * (1.0f - 4.5f * cu * cu + 1.5f * uu);
            float k = 3.0f + 9.0f * cu;  // dn^eq/dJ = w (3 c + 9 (c.u) c - 3 u)
            Bx += ws * (k * cx(m) - 3.0f * ux);
            By += ws * (k * cy(m) - 3.0f * uy);
            Bz += ws * (k * cz(m) - 3.0f * uz);
        }
        int x = (int)(L.coord[i] >> 20);
        float add = x == A.probe_x ? dl : 0.f;
#pragma unroll
        for (int j = 0; j < Q; ++j)
            out[(size_t)j * P + i] = (1.0f - om) * s[j] + om * (Aa + Bx * cx(j) + By * cy(j) + Bz * cz(j)) + add;
        dw = -(double)sw;
    }
    block_sum_to(dw, d_omega + blockIdx.x % GRAD_COPIES);
}

void launch_adj_step(const AdjArgs& A, const float* nat, float* out, float dl, double* d_omega, cudaStream_t s) {
    if (A.L.nS) k_adj_step<<<(A.L.nS + 255) / 256, 256, 0, s>>>(A, nat, out, dl, d_omega);
}

}  // namespace lbmdem
