// Assembly of the discrete pencil on the device (paper Sec. 4.2, App. A).
//
// Host side: index work only (P2 numbering, duplicated fluid-solid nodes,
// locality order, CSR patterns, per-element scatter positions, fluid-solid
// faces). Device side: element matrices in FP64 from reference-element
// matrices built the paper's way (Appendix A: generalized Vandermonde V of
// a monomial basis, mass = V^-T G V^-1 with G the monomial Gram matrix,
// derivative matrices D_j = (d_j V) V^-1), scattered with atomics into
// the resident CSR values; reference gravity by direct summation over
// tet point masses (Sec. 5.1).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "kernels.h"
#include "nm_internal.h"

namespace nm {

// ------------------------------------------------------------ reference element
struct RefMats {
    double M[100];          // int l_a l_b over the reference tet
    double D[3][100];       // nodal derivative matrices D_j[a][c]
    double S[3][3][100];    // int d_j l_a d_k l_b
    double C[3][100];       // int d_j l_a l_b
    double F[36];           // int l_a l_b over the reference triangle
};

__constant__ RefMats cRef;

static const int kEdge[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

static bool invert(int n, std::vector<double>& A) {   // Gauss-Jordan, partial pivoting
    std::vector<double> I(n * n, 0.0);
    for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[r * n + c]) > std::fabs(A[p * n + c])) p = r;
        if (std::fabs(A[p * n + c]) < 1e-14) return false;
        for (int k = 0; k < n; ++k) {
            std::swap(A[c * n + k], A[p * n + k]);
            std::swap(I[c * n + k], I[p * n + k]);
        }
        const double inv = 1.0 / A[c * n + c];
        for (int k = 0; k < n; ++k) {
            A[c * n + k] *= inv;
            I[c * n + k] *= inv;
        }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double f = A[r * n + c];
            if (f == 0.0) continue;
            for (int k = 0; k < n; ++k) {
                A[r * n + k] -= f * A[c * n + k];
                I[r * n + k] -= f * I[c * n + k];
            }
        }
    }
    A = I;
    return true;
}

static double fact(int k) {
    double f = 1;
    for (int i = 2; i <= k; ++i) f *= i;
    return f;
}

static int build_reference(RefMats& R) {
    // reference tet (0,0,0),(1,0,0),(0,1,0),(0,0,1); nodes: vertices then edge midpoints
    double node[10][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int e = 0; e < 6; ++e)
        for (int d = 0; d < 3; ++d)
            node[4 + e][d] = 0.5 * (node[kEdge[e][0]][d] + node[kEdge[e][1]][d]);
    const int ex[10][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0},
                           {0, 2, 0}, {0, 0, 2}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};
    auto mono = [&](int n, const double* x) {
        return std::pow(x[0], ex[n][0]) * std::pow(x[1], ex[n][1]) * std::pow(x[2], ex[n][2]);
    };
    auto dmono = [&](int n, int j, const double* x) {
        if (ex[n][j] == 0) return 0.0;
        double v = ex[n][j];
        for (int d = 0; d < 3; ++d) v *= std::pow(x[d], ex[n][d] - (d == j ? 1 : 0));
        return v;
    };
    std::vector<double> V(100), G(100);
    for (int i = 0; i < 10; ++i)
        for (int n = 0; n < 10; ++n) V[i * 10 + n] = mono(n, node[i]);
    for (int n = 0; n < 10; ++n)
        for (int p = 0; p < 10; ++p) {
            const int a = ex[n][0] + ex[p][0], b = ex[n][1] + ex[p][1], c = ex[n][2] + ex[p][2];
            G[n * 10 + p] = fact(a) * fact(b) * fact(c) / fact(a + b + c + 3);
        }
    std::vector<double> Vi = V;
    if (!invert(10, Vi)) return fail(NM_ECUDA, "reference Vandermonde matrix is singular");
    // M = Vi^T G Vi
    for (int a = 0; a < 10; ++a)
        for (int b = 0; b < 10; ++b) {
            double s = 0;
            for (int n = 0; n < 10; ++n)
                for (int p = 0; p < 10; ++p) s += Vi[n * 10 + a] * G[n * 10 + p] * Vi[p * 10 + b];
            R.M[a * 10 + b] = s;
        }
    for (int j = 0; j < 3; ++j)
        for (int a = 0; a < 10; ++a)
            for (int c = 0; c < 10; ++c) {
                double s = 0;
                for (int n = 0; n < 10; ++n) s += dmono(n, j, node[a]) * Vi[n * 10 + c];
                R.D[j][a * 10 + c] = s;
            }
    for (int j = 0; j < 3; ++j) {
        // C_j = D_j^T M
        for (int a = 0; a < 10; ++a)
            for (int b = 0; b < 10; ++b) {
                double s = 0;
                for (int c = 0; c < 10; ++c) s += R.D[j][c * 10 + a] * R.M[c * 10 + b];
                R.C[j][a * 10 + b] = s;
            }
        for (int k = 0; k < 3; ++k)
            for (int a = 0; a < 10; ++a)
                for (int b = 0; b < 10; ++b) {
                    double s = 0;
                    for (int c = 0; c < 10; ++c)
                        for (int d = 0; d < 10; ++d)
                            s += R.D[j][c * 10 + a] * R.M[c * 10 + d] * R.D[k][d * 10 + b];
                    R.S[j][k][a * 10 + b] = s;
                }
    }
    // reference triangle (0,0),(1,0),(0,1); nodes: vertices, edges (0,1),(0,2),(1,2)
    const double tn[6][2] = {{0, 0}, {1, 0}, {0, 1}, {0.5, 0}, {0, 0.5}, {0.5, 0.5}};
    const int te[6][2] = {{0, 0}, {1, 0}, {0, 1}, {2, 0}, {1, 1}, {0, 2}};
    std::vector<double> V2(36), G2(36);
    for (int i = 0; i < 6; ++i)
        for (int n = 0; n < 6; ++n)
            V2[i * 6 + n] = std::pow(tn[i][0], te[n][0]) * std::pow(tn[i][1], te[n][1]);
    for (int n = 0; n < 6; ++n)
        for (int p = 0; p < 6; ++p) {
            const int a = te[n][0] + te[p][0], b = te[n][1] + te[p][1];
            G2[n * 6 + p] = fact(a) * fact(b) / fact(a + b + 2);
        }
    if (!invert(6, V2)) return fail(NM_ECUDA, "reference triangle Vandermonde is singular");
    for (int a = 0; a < 6; ++a)
        for (int b = 0; b < 6; ++b) {
            double s = 0;
            for (int n = 0; n < 6; ++n)
                for (int p = 0; p < 6; ++p) s += V2[n * 6 + a] * G2[n * 6 + p] * V2[p * 6 + b];
            R.F[a * 6 + b] = s;
        }
    return NM_OK;
}

// ------------------------------------------------------------ device kernels
struct TetGeom {
    double detJ;          // |det J| (= 6 |K|)
    double Jinv[3][3];    // dr_j / dx_i stored as Jinv[j][i]
};

__device__ inline void tet_geom(const double* x, TetGeom& g) {
    double J[3][3];
    for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d) J[d][c] = x[3 * (c + 1) + d] - x[d];   // column c = x_{c+1} - x_0
    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    const double id = 1.0 / det;
    // inverse of J: r = J^{-1} (x - x0), so dr_j/dx_i = Jinv[j][i]
    g.Jinv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) * id;
    g.Jinv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
    g.Jinv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
    g.Jinv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) * id;
    g.Jinv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
    g.Jinv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
    g.Jinv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) * id;
    g.Jinv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
    g.Jinv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
    g.detJ = fabs(det);
}

struct ElemArgs {
    int64_t nt;
    const double* vx;       // [nt][4][3] vertex coordinates
    const int* unode;       // [nt][10] internal u-node ids
    const uint8_t* region;  // [nt]
    const double* rho;
    const double* lam;
    const double* mu;
    const double* N2;
    const double* g;        // [Nu][3] or nullptr
    const int* posU;        // [nt][100] positions in the u-graph
    double* AG;             // 9 per position
    double* Mr;             // 1 per position
};

// One block per tet; thread t < 100 owns the pair (a, b) = (t / 10, t % 10).
__global__ void __launch_bounds__(128) elem_u_kernel(const ElemArgs A) {
    const int64_t t = blockIdx.x;
    if (t >= A.nt) return;
    __shared__ TetGeom G;
    __shared__ double gn[10][3];
    __shared__ double dg[10][3][3];   // dg[a][i][j] = d_i g_j at node a
    const int tid = threadIdx.x;
    if (tid == 0) tet_geom(A.vx + 12 * t, G);
    const bool grav = A.g != nullptr;
    if (grav && tid < 30) {
        const int a = tid / 3, j = tid % 3;
        gn[a][j] = A.g[3 * (int64_t)A.unode[10 * t + a] + j];
    }
    __syncthreads();
    if (grav && tid < 90) {
        const int a = tid / 9, i = (tid / 3) % 3, j = tid % 3;
        double s = 0;
        for (int p = 0; p < 3; ++p) {
            double dj = 0;
            for (int c = 0; c < 10; ++c) dj += cRef.D[p][a * 10 + c] * gn[c][j];
            s += G.Jinv[p][i] * dj;
        }
        dg[a][i][j] = s;
    }
    __syncthreads();
    if (tid >= 100) return;
    const int a = tid / 10, b = tid % 10;
    const double dJ = G.detJ;
    const double rho = A.rho[t];
    const bool solid = A.region[t] == 0;
    const double mab = dJ * cRef.M[a * 10 + b];
    double K[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    if (solid) {
        double E[3][3];
        for (int p = 0; p < 3; ++p)
            for (int q = 0; q < 3; ++q) {
                double s = 0;
                for (int j = 0; j < 3; ++j)
                    for (int k = 0; k < 3; ++k) s += G.Jinv[j][p] * G.Jinv[k][q] * cRef.S[j][k][a * 10 + b];
                E[p][q] = dJ * s;      // int d_p phi_a d_q phi_b
            }
        const double lam = A.lam[t], mu = A.mu[t];
        const double tr = E[0][0] + E[1][1] + E[2][2];
        for (int m = 0; m < 3; ++m)
            for (int n = 0; n < 3; ++n) K[m][n] = lam * E[m][n] + mu * (E[n][m] + (m == n ? tr : 0.0));
    }
    if (grav) {
        if (solid) {
            double Cab[3], Cba[3];
            for (int m = 0; m < 3; ++m) {
                double s1 = 0, s2 = 0;
                for (int j = 0; j < 3; ++j) {
                    s1 += G.Jinv[j][m] * cRef.C[j][a * 10 + b];
                    s2 += G.Jinv[j][m] * cRef.C[j][b * 10 + a];
                }
                Cab[m] = dJ * s1;   // int d_m phi_a phi_b
                Cba[m] = dJ * s2;   // int d_m phi_b phi_a
            }
            for (int m = 0; m < 3; ++m)
                for (int n = 0; n < 3; ++n) {
                    // L[(a,m),(b,n)] = rho [C_a,m,b g_n(b) - d_m g_n(a) M_ab - C_a,n,b g_m(b)]
                    const double L = Cab[m] * gn[b][n] - dg[a][m][n] * mab - Cab[n] * gn[b][m];
                    // L[(b,n),(a,m)]
                    const double Lt = Cba[n] * gn[a][m] - dg[b][n][m] * mab - Cba[m] * gn[a][n];
                    K[m][n] += 0.5 * rho * (L + Lt);
                }
        } else {
            const double N2 = A.N2[t];
            double ha[3], hb[3];
            const double na = sqrt(gn[a][0] * gn[a][0] + gn[a][1] * gn[a][1] + gn[a][2] * gn[a][2]);
            const double nb = sqrt(gn[b][0] * gn[b][0] + gn[b][1] * gn[b][1] + gn[b][2] * gn[b][2]);
            for (int m = 0; m < 3; ++m) {
                ha[m] = na > 0 ? gn[a][m] / na : 0.0;
                hb[m] = nb > 0 ? gn[b][m] / nb : 0.0;
            }
            for (int m = 0; m < 3; ++m)
                for (int n = 0; n < 3; ++n) K[m][n] += rho * N2 * ha[m] * mab * hb[n];
        }
    }
    const int64_t pos = A.posU[100 * t + tid];
    for (int m = 0; m < 3; ++m)
        for (int n = 0; n < 3; ++n)
            if (K[m][n] != 0.0) atomicAdd(A.AG + 9 * pos + 3 * m + n, K[m][n]);
    atomicAdd(A.Mr + pos, rho * mab);
}

struct FluidArgs {
    int64_t nf;              // fluid tets
    const int64_t* tets;     // [nf] tet ids
    const double* vx;
    const int* unode;        // [nt][10]
    const double* rho;
    const double* lam;
    const double* mu;
    const double* g;         // or nullptr
    const int* posP;         // [nf][100] in the p-graph (p_a, p_b)
    const int* posE;         // [nf][100] in E_G (u_a, p_b)
    const int* posEt;        // [nf][100] in E_G^T (p_a, u_b)
    double* Pn;              // -A_p values
    double* EG;              // 3 per position
    double* EGt;             // 3 per position
};

__global__ void __launch_bounds__(128) elem_p_kernel(const FluidArgs A) {
    const int64_t f = blockIdx.x;
    if (f >= A.nf) return;
    const int64_t t = A.tets[f];
    __shared__ TetGeom G;
    __shared__ double gn[10][3];
    const int tid = threadIdx.x;
    if (tid == 0) tet_geom(A.vx + 12 * t, G);
    if (tid < 30) gn[tid / 3][tid % 3] = A.g ? A.g[3 * (int64_t)A.unode[10 * t + tid / 3] + tid % 3] : 0.0;
    __syncthreads();
    if (tid >= 100) return;
    const int a = tid / 10, b = tid % 10;
    const double dJ = G.detJ;
    const double kap = A.lam[t] + 2.0 * A.mu[t] / 3.0;
    const double rk = A.rho[t] / kap;
    const double mab = dJ * cRef.M[a * 10 + b];
    double Cab[3], Cba[3];
    for (int m = 0; m < 3; ++m) {
        double s1 = 0, s2 = 0;
        for (int j = 0; j < 3; ++j) {
            s1 += G.Jinv[j][m] * cRef.C[j][a * 10 + b];
            s2 += G.Jinv[j][m] * cRef.C[j][b * 10 + a];
        }
        Cab[m] = dJ * s1;
        Cba[m] = dJ * s2;
    }
    atomicAdd(A.Pn + A.posP[100 * f + tid], mab / kap);
    const int64_t pe = A.posE[100 * f + tid];
    const int64_t pt = A.posEt[100 * f + tid];
    for (int j = 0; j < 3; ++j) {
        // E_G[(u_a, j), p_b] = int phi_a d_j phi_b - rho/kappa g_j(a) M_ab
        atomicAdd(A.EG + 3 * pe + j, Cba[j] - rk * gn[a][j] * mab);
        // E_G^T[p_a, (u_b, j)] = E_G[(u_b, j), p_a]
        atomicAdd(A.EGt + 3 * pt + j, Cab[j] - rk * gn[b][j] * mab);
    }
}

struct FaceArgs {
    int64_t nfs;
    const double* nrm;      // [nfs][3] unit normal solid -> fluid
    const double* area;     // [nfs]
    const double* rho_f;    // [nfs] fluid density
    const int* us;          // [nfs][6] solid u-nodes
    const double* g;        // or nullptr
    const int* posU;        // [nfs][36] in the u-graph
    const int* posE;        // [nfs][36] in E_G (u_a, p_b)
    const int* posEt;       // [nfs][36] in E_G^T (p_a, u_b)
    double* AG;
    double* EG;
    double* EGt;
};

__global__ void face_kernel(const FaceArgs A) {
    const int64_t f = blockIdx.x;
    if (f >= A.nfs) return;
    const int tid = threadIdx.x;
    if (tid >= 36) return;
    const int a = tid / 6, b = tid % 6;
    const double fm = 2.0 * A.area[f] * cRef.F[a * 6 + b];
    const double* nu = A.nrm + 3 * f;
    const int64_t pe = A.posE[36 * f + tid];
    const int64_t pt = A.posEt[36 * f + tid];
    for (int j = 0; j < 3; ++j) {
        atomicAdd(A.EG + 3 * pe + j, nu[j] * fm);
        atomicAdd(A.EGt + 3 * pt + j, nu[j] * fm);
    }
    if (A.g) {
        const double* ga = A.g + 3 * (int64_t)A.us[6 * f + a];
        const double* gb = A.g + 3 * (int64_t)A.us[6 * f + b];
        const double rf = A.rho_f[f];
        const int64_t pu = A.posU[36 * f + tid];
        for (int m = 0; m < 3; ++m)
            for (int n = 0; n < 3; ++n)
                atomicAdd(A.AG + 9 * pu + 3 * m + n, 0.5 * rf * fm * (ga[m] * nu[n] + nu[m] * gb[n]));
    }
}

// g(x_i) = -G sum_k m_k (x_i - r_k) / |x_i - r_k|^3, sources staged in shared memory
__global__ void __launch_bounds__(256) gravity_kernel(int64_t nx, const double* x, int64_t ns,
                                                      const double* src /* [ns][4]: r, m */,
                                                      double G, double* g) {
    __shared__ double sh[256][4];
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double xi0 = 0, xi1 = 0, xi2 = 0;
    if (i < nx) {
        xi0 = x[3 * i];
        xi1 = x[3 * i + 1];
        xi2 = x[3 * i + 2];
    }
    double a0 = 0, a1 = 0, a2 = 0;
    for (int64_t s0 = 0; s0 < ns; s0 += 256) {
        const int64_t sk = s0 + threadIdx.x;
        for (int d = 0; d < 4; ++d) sh[threadIdx.x][d] = sk < ns ? src[4 * sk + d] : 0.0;
        __syncthreads();
        const int cnt = (int)((ns - s0) < 256 ? (ns - s0) : 256);
        for (int k = 0; k < cnt; ++k) {
            const double d0 = xi0 - sh[k][0], d1 = xi1 - sh[k][1], d2 = xi2 - sh[k][2];
            const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
            const double ir = rsqrt(r2);
            const double w = sh[k][3] * ir * ir * ir;
            a0 += w * d0;
            a1 += w * d1;
            a2 += w * d2;
        }
        __syncthreads();
    }
    if (i < nx) {
        g[3 * i] = -G * a0;
        g[3 * i + 1] = -G * a1;
        g[3 * i + 2] = -G * a2;
    }
}

__global__ void dinv_kernel(int64_t n, const double* val, const int64_t* dpos, double* dinv,
                            float* dinv32) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = 1.0 / val[dpos[i]];
        dinv[i] = v;
        dinv32[i] = (float)v;
    }
}

// ------------------------------------------------------------ host helpers
static uint64_t spread3(uint64_t v) {
    v &= 0x1fffff;
    v = (v | v << 32) & 0x1f00000000ffffULL;
    v = (v | v << 16) & 0x1f0000ff0000ffULL;
    v = (v | v << 8) & 0x100f00f00f00f00fULL;
    v = (v | v << 4) & 0x10c30c30c30c30c3ULL;
    v = (v | v << 2) & 0x1249249249249249ULL;
    return v;
}

// A group of "elements" each connecting `nr` row nodes with `nc` column nodes.
struct ElemGroup {
    int64_t count;
    int nr, nc;
    const int* rows;   // [count][nr]
    const int* cols;   // [count][nc]
};

// CSR pattern (sorted columns) of the union of all element couplings.
static int build_pattern(int64_t nrows, const std::vector<ElemGroup>& groups,
                         std::vector<int32_t>& rowptr, std::vector<int32_t>& col) {
    // incidence: row node -> (group, element)
    std::vector<int64_t> cnt(nrows + 1, 0);
    for (auto& g : groups)
        for (int64_t e = 0; e < g.count; ++e)
            for (int a = 0; a < g.nr; ++a) cnt[g.rows[e * g.nr + a] + 1]++;
    for (int64_t i = 0; i < nrows; ++i) cnt[i + 1] += cnt[i];
    std::vector<int64_t> inc(cnt[nrows]);
    std::vector<int> ginc(cnt[nrows]);
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (size_t gi = 0; gi < groups.size(); ++gi) {
        auto& g = groups[gi];
        for (int64_t e = 0; e < g.count; ++e)
            for (int a = 0; a < g.nr; ++a) {
                const int64_t r = g.rows[e * g.nr + a];
                inc[fill[r]] = e;
                ginc[fill[r]] = (int)gi;
                fill[r]++;
            }
    }
    std::vector<std::vector<int32_t>> rowcols(nrows);
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t r = 0; r < nrows; ++r) {
        auto& v = rowcols[r];
        for (int64_t q = cnt[r]; q < cnt[r + 1]; ++q) {
            const auto& g = groups[ginc[q]];
            const int64_t e = inc[q];
            for (int b = 0; b < g.nc; ++b) v.push_back(g.cols[e * g.nc + b]);
        }
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
    }
    rowptr.assign(nrows + 1, 0);
    int64_t total = 0;
    for (int64_t r = 0; r < nrows; ++r) {
        total += (int64_t)rowcols[r].size();
        if (total > INT32_MAX) return fail(NM_EUNSUPPORTED, "sparse pattern exceeds 2^31 entries");
        rowptr[r + 1] = (int32_t)total;
    }
    col.resize(total);
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t r = 0; r < nrows; ++r)
        std::copy(rowcols[r].begin(), rowcols[r].end(), col.begin() + rowptr[r]);
    return NM_OK;
}

static void scatter_positions(const std::vector<int32_t>& rowptr, const std::vector<int32_t>& col,
                              const ElemGroup& g, std::vector<int32_t>& pos) {
    pos.resize(g.count * g.nr * g.nc);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < g.count; ++e)
        for (int a = 0; a < g.nr; ++a) {
            const int r = g.rows[e * g.nr + a];
            const int32_t* b0 = col.data() + rowptr[r];
            const int32_t* b1 = col.data() + rowptr[r + 1];
            for (int b = 0; b < g.nc; ++b) {
                const int c = g.cols[e * g.nc + b];
                pos[(e * g.nr + a) * g.nc + b] = (int32_t)(std::lower_bound(b0, b1, c) - col.data());
            }
        }
}

template <class T>
static int upload(DevBuf& buf, const std::vector<T>& h) {
    NM_TRY(buf.alloc(std::max<size_t>(h.size(), 1) * sizeof(T)));
    if (!h.empty()) NM_CUDA(cudaMemcpy(buf.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return NM_OK;
}

static int upload_pattern(DevCSR& A, int64_t nrows, int64_t ncols, int rb, int cb,
                          std::vector<int32_t>&& rp, std::vector<int32_t>&& col) {
    A.nrows = nrows;
    A.ncols = ncols;
    A.nnz = rp.empty() ? 0 : rp.back();
    A.rb = rb;
    A.cb = cb;
    NM_TRY(upload(A.rowptr, rp));
    NM_TRY(upload(A.col, col));
    NM_TRY(A.val.alloc(std::max<int64_t>(A.nnz, 1) * rb * cb * sizeof(double)));
    NM_CUDA(cudaMemset(A.val.p, 0, std::max<int64_t>(A.nnz, 1) * rb * cb * sizeof(double)));
    A.h_rowptr = std::move(rp);
    A.h_col = std::move(col);
    return NM_OK;
}

// Row tiles of a scalar square pattern (see DevCSR): the distinct columns of
// each tile of `rows` consecutive rows and every entry's local position.
static int build_tiles(DevCSR& A, int rows) {
    const int64_t n = A.nrows;
    A.tile_rows = rows;
    A.ntiles = (n + rows - 1) / rows;
    std::vector<int32_t> uptr(A.ntiles + 1, 0), ucol;
    std::vector<uint16_t> lcol(std::max<int64_t>(A.nnz, 1));
    ucol.reserve((size_t)n * 6);
    int umax = 0;
    std::vector<int32_t> tmp;
    for (int64_t t = 0; t < A.ntiles; ++t) {
        const int64_t r0 = t * rows, r1 = std::min<int64_t>(n, r0 + rows);
        tmp.assign(A.h_col.begin() + A.h_rowptr[r0], A.h_col.begin() + A.h_rowptr[r1]);
        std::sort(tmp.begin(), tmp.end());
        tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
        if (tmp.size() > 65535) return fail(NM_EUNSUPPORTED, "tile with more than 65535 distinct columns");
        umax = std::max<int>(umax, (int)tmp.size());
        for (int64_t e = A.h_rowptr[r0]; e < A.h_rowptr[r1]; ++e)
            lcol[e] = (uint16_t)(std::lower_bound(tmp.begin(), tmp.end(), A.h_col[e]) - tmp.begin());
        ucol.insert(ucol.end(), tmp.begin(), tmp.end());
        uptr[t + 1] = (int32_t)ucol.size();
    }
    A.tile_umax = umax;
    NM_TRY(upload(A.tile_uptr, uptr));
    NM_TRY(upload(A.tile_ucol, ucol));
    NM_TRY(upload(A.lcol, lcol));
    return NM_OK;
}

int set_tile_rows(nm_problem* P, int64_t rows) {
    if (rows == 0) {
        for (DevCSR* A : {&P->Mr, &P->Pn}) {
            A->tile_uptr.release();
            A->tile_ucol.release();
            A->lcol.release();
            A->tile_rows = 0;
            A->ntiles = 0;
            A->tile_umax = 0;
        }
        return NM_OK;
    }
    if (rows < 4 || rows > 64 || (rows & (rows - 1))) return fail(NM_EINVAL, "tile_rows must be 0 or 4..64, a power of two");
    NM_TRY(build_tiles(P->Mr, (int)rows));
    if (P->info.Np > 0) NM_TRY(build_tiles(P->Pn, (int)rows));
    if ((size_t)P->Mr.tile_umax * 3 * 32 * sizeof(float) > 200 * 1024)
        return fail(NM_EINVAL, "tile_rows too large: staged operand exceeds shared memory");
    return NM_OK;
}

// ------------------------------------------------------------ nm_assemble
int assemble(nm_ctx* ctx, const nm_mesh* mesh, const nm_model* mdl, nm_problem* P) {
    const int64_t nv = mesh->nv, nt = mesh->nt;
    if (nv < 4 || nt < 1 || !mesh->xyz || !mesh->tet || !mesh->region)
        return fail(NM_EINVAL, "mesh needs nv >= 4, nt >= 1 and non-null arrays");
    if (nv > INT32_MAX / 8 || nt > INT32_MAX / 128) return fail(NM_EUNSUPPORTED, "mesh too large for int32 indices");
    if (!mdl || !mdl->rho || !mdl->lam || !mdl->mu) return fail(NM_EINVAL, "model arrays rho, lam, mu are required");
    if (mdl->flags & NM_CENTRIFUGAL) return fail(NM_EUNSUPPORTED, "centrifugal term is not supported");
    const bool gravity = (mdl->flags & NM_GRAVITY) != 0;
    const int32_t* tet = mesh->tet;
    const double* xyz = mesh->xyz;
    // ---- validation
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t v = 0; v < nv; ++v)
        for (int d = 0; d < 3; ++d) {
            const double x = xyz[3 * v + d];
            if (!std::isfinite(x)) return fail(NM_EINVAL, "non-finite vertex coordinate");
            lo[d] = std::min(lo[d], x);
            hi[d] = std::max(hi[d], x);
        }
    const double diam = std::sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                                  (hi[2] - lo[2]) * (hi[2] - lo[2]));
    int64_t nfluid = 0;
    for (int64_t t = 0; t < nt; ++t) {
        for (int a = 0; a < 4; ++a)
            if (tet[4 * t + a] < 0 || tet[4 * t + a] >= nv) return fail(NM_EINVAL, "tet vertex id out of range");
        const uint8_t r = mesh->region[t];
        if (r > 1) return fail(NM_EINVAL, "region must be 0 (solid) or 1 (fluid)");
        if (!(mdl->rho[t] > 0)) return fail(NM_EINVAL, "rho must be positive");
        const double kap = mdl->lam[t] + 2.0 * mdl->mu[t] / 3.0;
        if (!(kap > 0) || !(mdl->mu[t] >= 0)) return fail(NM_EINVAL, "need mu >= 0 and kappa > 0");
        if (r == 1) {
            if (mdl->mu[t] != 0.0) return fail(NM_EINVAL, "fluid tets need mu = 0");
            ++nfluid;
        }
        const double* x0 = xyz + 3 * tet[4 * t];
        double J[3][3];
        for (int c = 0; c < 3; ++c)
            for (int d = 0; d < 3; ++d) J[c][d] = xyz[3 * tet[4 * t + c + 1] + d] - x0[d];
        const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                           J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                           J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        if (!(std::fabs(det) > 1e-13 * diam * diam * diam)) return fail(NM_EINVAL, "degenerate tetrahedron");
    }
    if (nfluid > 0 && (!mdl->N2 && gravity)) return fail(NM_EINVAL, "N2 is required with fluid tets and gravity");
    RefMats R;
    NM_TRY(build_reference(R));
    NM_CUDA(cudaMemcpyToSymbol(cRef, &R, sizeof(RefMats)));

    // ---- P2 nodes: vertices then edges in lexicographic (min, max) order
    std::vector<int64_t> ekey(6 * nt);
    for (int64_t t = 0; t < nt; ++t)
        for (int e = 0; e < 6; ++e) {
            int64_t a = tet[4 * t + kEdge[e][0]], b = tet[4 * t + kEdge[e][1]];
            if (a > b) std::swap(a, b);
            if (a == b) return fail(NM_EINVAL, "tet with repeated vertex");
            ekey[6 * t + e] = a * nv + b;
        }
    std::vector<int64_t> ukey(ekey);
    std::sort(ukey.begin(), ukey.end());
    ukey.erase(std::unique(ukey.begin(), ukey.end()), ukey.end());
    const int64_t ne = (int64_t)ukey.size();
    const int64_t n_p2 = nv + ne;
    std::vector<int64_t> tet10(10 * nt);
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < nt; ++t) {
        for (int a = 0; a < 4; ++a) tet10[10 * t + a] = tet[4 * t + a];
        for (int e = 0; e < 6; ++e)
            tet10[10 * t + 4 + e] =
                nv + (std::lower_bound(ukey.begin(), ukey.end(), ekey[6 * t + e]) - ukey.begin());
    }
    std::vector<double> pxyz(3 * n_p2);
    std::copy(xyz, xyz + 3 * nv, pxyz.begin());
    for (int64_t e = 0; e < ne; ++e) {
        const int64_t a = ukey[e] / nv, b = ukey[e] % nv;
        for (int d = 0; d < 3; ++d) pxyz[3 * (nv + e) + d] = 0.5 * (xyz[3 * a + d] + xyz[3 * b + d]);
    }
    // ---- canonical u-nodes (solid copies, then fluid copies) and p-nodes
    std::vector<uint8_t> touch(n_p2, 0);   // bit 0 solid, bit 1 fluid
    for (int64_t t = 0; t < nt; ++t)
        for (int a = 0; a < 10; ++a) touch[tet10[10 * t + a]] |= (mesh->region[t] ? 2 : 1);
    std::vector<int64_t> us(n_p2, -1), uf(n_p2, -1);
    int64_t ns = 0, nfn = 0;
    for (int64_t q = 0; q < n_p2; ++q)
        if (touch[q] & 1) us[q] = ns++;
    for (int64_t q = 0; q < n_p2; ++q)
        if (touch[q] & 2) uf[q] = ns + nfn++;
    const int64_t Nu = ns + nfn, Np = nfn;
    std::vector<int64_t> u_p2(Nu);
    for (int64_t q = 0; q < n_p2; ++q) {
        if (us[q] >= 0) u_p2[us[q]] = q;
        if (uf[q] >= 0) u_p2[uf[q]] = q;
    }
    // ---- locality order: Morton code of the node position (ties by canonical id)
    std::vector<uint64_t> code(Nu);
    for (int64_t u = 0; u < Nu; ++u) {
        uint64_t c = 0;
        for (int d = 0; d < 3; ++d) {
            const double s = hi[d] > lo[d] ? (pxyz[3 * u_p2[u] + d] - lo[d]) / (hi[d] - lo[d]) : 0.0;
            const uint64_t qd = (uint64_t)std::min(2097151.0, std::max(0.0, s * 2097151.0));
            c |= spread3(qd) << d;
        }
        code[u] = c;
    }
    std::vector<int64_t> order(Nu);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return code[a] < code[b]; });
    std::vector<int32_t> int_of_can(Nu);
    for (int64_t i = 0; i < Nu; ++i) int_of_can[order[i]] = (int32_t)i;
    P->canon_of_internal = order;
    P->p2_of_internal.resize(Nu);
    for (int64_t i = 0; i < Nu; ++i) P->p2_of_internal[i] = u_p2[order[i]];
    // internal p order follows the internal order of the fluid copies
    std::vector<int32_t> pint_of_p2(n_p2, -1);
    P->pcanon_of_internal.clear();
    for (int64_t i = 0; i < Nu; ++i) {
        const int64_t c = order[i];
        if (c >= ns) {
            pint_of_p2[u_p2[c]] = (int32_t)P->pcanon_of_internal.size();
            P->pcanon_of_internal.push_back(c - ns);
        }
    }
    // ---- per-tet internal u-nodes
    std::vector<int32_t> tu(10 * nt);
    for (int64_t t = 0; t < nt; ++t)
        for (int a = 0; a < 10; ++a) {
            const int64_t q = tet10[10 * t + a];
            tu[10 * t + a] = int_of_can[mesh->region[t] ? uf[q] : us[q]];
        }
    // ---- fluid-solid faces
    std::vector<int64_t> fs_ts, fs_tf;
    std::vector<int32_t> fs_tri;   // vertex ids in the solid tet's order
    if (nfluid > 0 && nfluid < nt) {
        static const int fv[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
        struct F { int64_t k0, k1; int64_t t; int loc; };
        std::vector<F> faces(4 * nt);
        for (int64_t t = 0; t < nt; ++t)
            for (int f = 0; f < 4; ++f) {
                int64_t v[3] = {tet[4 * t + fv[f][0]], tet[4 * t + fv[f][1]], tet[4 * t + fv[f][2]]};
                std::sort(v, v + 3);
                faces[4 * t + f] = {v[0] * nv + v[1], v[2], t, f};
            }
        std::sort(faces.begin(), faces.end(), [](const F& a, const F& b) {
            return a.k0 != b.k0 ? a.k0 < b.k0 : (a.k1 != b.k1 ? a.k1 < b.k1 : a.t < b.t);
        });
        for (size_t i = 0; i + 1 < faces.size(); ++i) {
            if (faces[i].k0 == faces[i + 1].k0 && faces[i].k1 == faces[i + 1].k1) {
                if (i + 2 < faces.size() && faces[i + 2].k0 == faces[i].k0 && faces[i + 2].k1 == faces[i].k1)
                    return fail(NM_EINVAL, "face shared by more than two tets");
                const F& A = faces[i];
                const F& B = faces[i + 1];
                const uint8_t ra = mesh->region[A.t], rb = mesh->region[B.t];
                if (ra != rb) {
                    const F& S = ra == 0 ? A : B;
                    const F& Fl = ra == 0 ? B : A;
                    fs_ts.push_back(S.t);
                    fs_tf.push_back(Fl.t);
                    for (int k = 0; k < 3; ++k) fs_tri.push_back(tet[4 * S.t + fv[S.loc][k]]);
                    fs_tri.push_back(tet[4 * S.t + S.loc]);   // opposite vertex (orientation)
                }
                ++i;
            }
        }
    }
    const int64_t nfs = (int64_t)fs_ts.size();
    std::vector<int32_t> fs_us(6 * nfs), fs_p(6 * nfs);
    std::vector<double> fs_n(3 * nfs), fs_a(nfs), fs_rho(nfs);
    for (int64_t f = 0; f < nfs; ++f) {
        const int32_t* tri = &fs_tri[4 * f];
        const int64_t ts = fs_ts[f];
        int64_t q[6];
        for (int k = 0; k < 3; ++k) q[k] = tri[k];
        const int fe[3][2] = {{0, 1}, {0, 2}, {1, 2}};
        for (int k = 0; k < 3; ++k) {
            int64_t a = tri[fe[k][0]], b = tri[fe[k][1]];
            if (a > b) std::swap(a, b);
            q[3 + k] = nv + (std::lower_bound(ukey.begin(), ukey.end(), a * nv + b) - ukey.begin());
        }
        for (int k = 0; k < 6; ++k) {
            fs_us[6 * f + k] = int_of_can[us[q[k]]];
            fs_p[6 * f + k] = pint_of_p2[q[k]];
        }
        const double* p0 = xyz + 3 * tri[0];
        const double* p1 = xyz + 3 * tri[1];
        const double* p2 = xyz + 3 * tri[2];
        const double* po = xyz + 3 * tri[3];
        double u[3], v[3], nn[3];
        for (int d = 0; d < 3; ++d) {
            u[d] = p1[d] - p0[d];
            v[d] = p2[d] - p0[d];
        }
        nn[0] = u[1] * v[2] - u[2] * v[1];
        nn[1] = u[2] * v[0] - u[0] * v[2];
        nn[2] = u[0] * v[1] - u[1] * v[0];
        const double len = std::sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
        double side = 0;
        for (int d = 0; d < 3; ++d) side += (po[d] - p0[d]) * nn[d];
        const double sg = side > 0 ? -1.0 : 1.0;   // away from the solid tet
        for (int d = 0; d < 3; ++d) fs_n[3 * f + d] = sg * nn[d] / len;
        fs_a[f] = 0.5 * len;
        fs_rho[f] = mdl->rho[fs_tf[f]];
        (void)ts;
    }
    // ---- patterns and scatter positions
    ElemGroup gt{nt, 10, 10, tu.data(), tu.data()};
    std::vector<int32_t> rp, cl;
    NM_TRY(build_pattern(Nu, {gt}, rp, cl));
    std::vector<int32_t> posU, posFU;
    scatter_positions(rp, cl, gt, posU);
    ElemGroup gf{nfs, 6, 6, fs_us.data(), fs_us.data()};
    if (nfs) scatter_positions(rp, cl, gf, posFU);
    std::vector<int32_t> rp2(rp), cl2(cl);
    NM_TRY(upload_pattern(P->AG, Nu, Nu, 3, 3, std::move(rp), std::move(cl)));
    NM_TRY(upload_pattern(P->Mr, Nu, Nu, 1, 1, std::move(rp2), std::move(cl2)));

    std::vector<int64_t> ftets;
    std::vector<int32_t> ftu, ftp;   // fluid tets: u-nodes and p-nodes
    for (int64_t t = 0; t < nt; ++t)
        if (mesh->region[t]) {
            ftets.push_back(t);
            for (int a = 0; a < 10; ++a) {
                ftu.push_back(tu[10 * t + a]);
                ftp.push_back(pint_of_p2[tet10[10 * t + a]]);
            }
        }
    const int64_t nft = (int64_t)ftets.size();
    std::vector<int32_t> posP, posE, posEt, posFE, posFEt;
    if (Np > 0) {
        ElemGroup gpp{nft, 10, 10, ftp.data(), ftp.data()};
        ElemGroup gup{nft, 10, 10, ftu.data(), ftp.data()};
        ElemGroup gpu{nft, 10, 10, ftp.data(), ftu.data()};
        ElemGroup gfup{nfs, 6, 6, fs_us.data(), fs_p.data()};
        ElemGroup gfpu{nfs, 6, 6, fs_p.data(), fs_us.data()};
        std::vector<int32_t> a, b;
        NM_TRY(build_pattern(Np, {gpp}, a, b));
        scatter_positions(a, b, gpp, posP);
        NM_TRY(upload_pattern(P->Pn, Np, Np, 1, 1, std::move(a), std::move(b)));
        std::vector<int32_t> c, d;
        NM_TRY(build_pattern(Nu, {gup, gfup}, c, d));
        scatter_positions(c, d, gup, posE);
        if (nfs) scatter_positions(c, d, gfup, posFE);
        NM_TRY(upload_pattern(P->EG, Nu, Np, 3, 1, std::move(c), std::move(d)));
        std::vector<int32_t> e, f;
        NM_TRY(build_pattern(Np, {gpu, gfpu}, e, f));
        scatter_positions(e, f, gpu, posEt);
        if (nfs) scatter_positions(e, f, gfpu, posFEt);
        NM_TRY(upload_pattern(P->EGt, Np, Nu, 1, 3, std::move(e), std::move(f)));
    }

    // ---- device inputs
    cudaStream_t s = ctx->stream;
    DevBuf d_vx, d_tu, d_reg, d_rho, d_lam, d_mu, d_N2, d_posU;
    std::vector<double> vx(12 * nt);
    for (int64_t t = 0; t < nt; ++t)
        for (int a = 0; a < 4; ++a)
            for (int d = 0; d < 3; ++d) vx[12 * t + 3 * a + d] = xyz[3 * tet[4 * t + a] + d];
    NM_TRY(upload(d_vx, vx));
    NM_TRY(upload(d_tu, tu));
    NM_TRY(upload(d_reg, std::vector<uint8_t>(mesh->region, mesh->region + nt)));
    NM_TRY(upload(d_rho, std::vector<double>(mdl->rho, mdl->rho + nt)));
    NM_TRY(upload(d_lam, std::vector<double>(mdl->lam, mdl->lam + nt)));
    NM_TRY(upload(d_mu, std::vector<double>(mdl->mu, mdl->mu + nt)));
    NM_TRY(upload(d_N2, mdl->N2 ? std::vector<double>(mdl->N2, mdl->N2 + nt) : std::vector<double>(nt, 0.0)));
    NM_TRY(upload(d_posU, posU));

    // ---- reference field g' at the u-nodes
    NM_TRY(P->g.alloc(3 * Nu * sizeof(double)));
    NM_CUDA(cudaMemsetAsync(P->g.p, 0, 3 * Nu * sizeof(double), s));
    if (gravity) {
        if (mdl->gprime) {
            std::vector<double> gh(3 * Nu);
            for (int64_t i = 0; i < Nu; ++i)
                for (int d = 0; d < 3; ++d) gh[3 * i + d] = mdl->gprime[3 * P->p2_of_internal[i] + d];
            NM_CUDA(cudaMemcpy(P->g.p, gh.data(), gh.size() * sizeof(double), cudaMemcpyHostToDevice));
        } else {
            std::vector<double> ux(3 * Nu), src(4 * nt);
            for (int64_t i = 0; i < Nu; ++i)
                for (int d = 0; d < 3; ++d) ux[3 * i + d] = pxyz[3 * P->p2_of_internal[i] + d];
            for (int64_t t = 0; t < nt; ++t) {
                double c[3] = {0, 0, 0};
                for (int a = 0; a < 4; ++a)
                    for (int d = 0; d < 3; ++d) c[d] += 0.25 * vx[12 * t + 3 * a + d];
                const double* x = &vx[12 * t];
                double J[3][3];
                for (int cc = 0; cc < 3; ++cc)
                    for (int d = 0; d < 3; ++d) J[cc][d] = x[3 * (cc + 1) + d] - x[d];
                const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                                   J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                                   J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
                for (int d = 0; d < 3; ++d) src[4 * t + d] = c[d];
                src[4 * t + 3] = mdl->rho[t] * std::fabs(det) / 6.0;
            }
            DevBuf d_ux, d_src;
            NM_TRY(upload(d_ux, ux));
            NM_TRY(upload(d_src, src));
            gravity_kernel<<<(unsigned)((Nu + 255) / 256), 256, 0, s>>>(Nu, d_ux.as<double>(), nt,
                                                                       d_src.as<double>(), mdl->G,
                                                                       P->g.as<double>());
            count_launch();
        NM_CUDA(cudaGetLastError());
            NM_CUDA(cudaStreamSynchronize(s));
        }
    }

    // ---- element kernels
    ElemArgs ea{nt, d_vx.as<double>(), d_tu.as<int>(), d_reg.as<uint8_t>(), d_rho.as<double>(),
                d_lam.as<double>(), d_mu.as<double>(), d_N2.as<double>(),
                gravity ? P->g.as<double>() : nullptr, d_posU.as<int>(), P->AG.val.as<double>(),
                P->Mr.val.as<double>()};
    elem_u_kernel<<<(unsigned)nt, 128, 0, s>>>(ea);
    count_launch();
        NM_CUDA(cudaGetLastError());
    DevBuf d_ftets, d_posP, d_posE, d_posEt, d_fn, d_fa, d_frho, d_fus, d_posFU, d_posFE, d_posFEt;
    if (Np > 0) {
        NM_TRY(upload(d_ftets, ftets));
        NM_TRY(upload(d_posP, posP));
        NM_TRY(upload(d_posE, posE));
        NM_TRY(upload(d_posEt, posEt));
        FluidArgs fa{nft, d_ftets.as<int64_t>(), d_vx.as<double>(), d_tu.as<int>(), d_rho.as<double>(),
                     d_lam.as<double>(), d_mu.as<double>(), gravity ? P->g.as<double>() : nullptr,
                     d_posP.as<int>(), d_posE.as<int>(), d_posEt.as<int>(), P->Pn.val.as<double>(),
                     P->EG.val.as<double>(), P->EGt.val.as<double>()};
        elem_p_kernel<<<(unsigned)nft, 128, 0, s>>>(fa);
        count_launch();
        NM_CUDA(cudaGetLastError());
        if (nfs > 0) {
            NM_TRY(upload(d_fn, fs_n));
            NM_TRY(upload(d_fa, fs_a));
            NM_TRY(upload(d_frho, fs_rho));
            NM_TRY(upload(d_fus, fs_us));
            NM_TRY(upload(d_posFU, posFU));
            NM_TRY(upload(d_posFE, posFE));
            NM_TRY(upload(d_posFEt, posFEt));
            FaceArgs fc{nfs, d_fn.as<double>(), d_fa.as<double>(), d_frho.as<double>(), d_fus.as<int>(),
                        gravity ? P->g.as<double>() : nullptr, d_posFU.as<int>(), d_posFE.as<int>(),
                        d_posFEt.as<int>(), P->AG.val.as<double>(), P->EG.val.as<double>(),
                        P->EGt.val.as<double>()};
            face_kernel<<<(unsigned)nfs, 64, 0, s>>>(fc);
            count_launch();
        NM_CUDA(cudaGetLastError());
        }
    }
    // ---- inverse diagonals of M_rho and -A_p
    auto make_dinv = [&](DevCSR& A) -> int {
        std::vector<int64_t> dpos(A.nrows);
        for (int64_t i = 0; i < A.nrows; ++i) {
            const int32_t* b0 = A.h_col.data() + A.h_rowptr[i];
            const int32_t* b1 = A.h_col.data() + A.h_rowptr[i + 1];
            const int32_t* it = std::lower_bound(b0, b1, (int32_t)i);
            if (it == b1 || *it != i) return fail(NM_EINVAL, "matrix row without a diagonal entry");
            dpos[i] = it - A.h_col.data();
        }
        DevBuf d_dpos;
        NM_TRY(upload(d_dpos, dpos));
        NM_TRY(A.dinv.alloc(std::max<int64_t>(A.nrows, 1) * sizeof(double)));
        NM_TRY(A.dinv32.alloc(std::max<int64_t>(A.nrows, 1) * sizeof(float)));
        dinv_kernel<<<(unsigned)std::min<int64_t>((A.nrows + 255) / 256 + 1, 4096), 256, 0, s>>>(
            A.nrows, A.val.as<double>(), d_dpos.as<int64_t>(), A.dinv.as<double>(), A.dinv32.as<float>());
        count_launch();
        NM_CUDA(cudaGetLastError());
        NM_CUDA(cudaStreamSynchronize(s));
        return NM_OK;
    };
    NM_CUDA(cudaStreamSynchronize(s));
    NM_TRY(make_dinv(P->Mr));
    if (Np > 0) NM_TRY(make_dinv(P->Pn));
    // region counters of the SM-local schedule (one per SM)
    {
        int dev = 0, sms = 0;
        NM_CUDA(cudaGetDevice(&dev));
        NM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        P->nreg = sms > 0 ? sms : 1;
        NM_TRY(P->sched.alloc((size_t)P->nreg * sizeof(int)));
    }
    NM_CUDA(cudaStreamSynchronize(s));

    auto& I = P->info;
    I.nv = nv;
    I.nt = nt;
    I.n_p2 = n_p2;
    I.Nu = Nu;
    I.n = 3 * Nu;
    I.Np = Np;
    I.nnz_u = P->AG.nnz;
    I.nnz_p = P->Pn.nnz;
    I.nnz_e = P->EG.nnz;
    I.n_fs = nfs;
    P->flags = mdl->flags;
    for (int d = 0; d < 3; ++d) P->Omega[d] = mdl->Omega[d];
    if (mdl->flags & NM_SELF_GRAVITY) {
        std::vector<int32_t> usol(n_p2, -1), uflu(n_p2, -1);
        for (int64_t q = 0; q < n_p2; ++q) {
            if (us[q] >= 0) usol[q] = int_of_can[us[q]];
            if (uf[q] >= 0) uflu[q] = int_of_can[uf[q]];
        }
        NM_TRY(nm::build_self_gravity(P, xyz, tet, tet10.data(), mesh->region, mdl->rho, nt, usol.data(),
                                      uflu.data(), mdl->G));
        I.n_charges = P->sg.np;
    }
    return NM_OK;
}

__global__ void lo_part_kernel(int64_t n, const double* v, const float* hi, float* lo) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        lo[t] = __double2float_rn(v[t] - (double)hi[t]);
}

int ensure_f32(nm_problem* P, cudaStream_t s);

// Low float parts of the matrix values for the double-float kernels.
int ensure_df(nm_problem* P, cudaStream_t s) {
    NM_TRY(ensure_f32(P, s));
    for (DevCSR* A : {&P->AG, &P->Mr, &P->Pn}) {
        if (A->nnz == 0 || A->vlo32.p) continue;
        const int64_t cnt = A->nnz * A->rb * A->cb;
        NM_TRY(A->vlo32.alloc(cnt * sizeof(float)));
        lo_part_kernel<<<(unsigned)std::min<int64_t>((cnt + 255) / 256, 4864), 256, 0, s>>>(
            cnt, A->val.as<double>(), A->val32.as<float>(), A->vlo32.as<float>());
        count_launch();
        NM_CUDA(cudaGetLastError());
    }
    return NM_OK;
}

// Float copies of the matrix values (created on first FP32 use).
int ensure_f32(nm_problem* P, cudaStream_t s) {
    auto conv = [&](DevCSR& A) -> int {
        if (A.nnz == 0 || A.val32.p) return NM_OK;
        const int64_t cnt = A.nnz * A.rb * A.cb;
        NM_TRY(A.val32.alloc(cnt * sizeof(float)));
        NM_TRY(launch_d2f(cnt, A.val.as<double>(), A.val32.as<float>(), s));
        return NM_OK;
    };
    NM_TRY(conv(P->AG));
    NM_TRY(conv(P->Mr));
    NM_TRY(conv(P->Pn));
    NM_TRY(conv(P->EG));
    NM_TRY(conv(P->EGt));
    return NM_OK;
}

}  // namespace nm
