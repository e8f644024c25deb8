// Self-gravitation: the term -C^T S C of the full operator (Sec. 5.2,
// eqs. ph1body2, ph1surface2, phi1fluidsolid, eigfull).
//
// The potential perturbation S(u) comes from point masses at the
// barycentres of the elements and of the charged faces: an element carries
// rho_k int_K div u, an outer face -rho_inside int_E (nu . u) (nu outward),
// a fluid-solid face rho_f int_E (nu . u^f) - rho_s int_E (nu . u^s) (nu
// from solid to fluid, each side's own copy of the interface nodes), and a
// face between two tets of one region whose per-element densities differ
// (rho_+ - rho_-) int_E (nu . u) (nu from - to +), the surface part of
// div(rho u) for the piecewise-constant density. With P2 shape functions an
// element charge involves its edge nodes only (int_K grad(4 l_a l_b) =
// |K| (grad l_a + grad l_b); the vertex functions integrate to zero), and a
// face charge its edge nodes with weight |E|/3. The potential at point i is
// G sum_{j != i} q_j / |r_i - r_j| + G q_i / R_i with
// 1/R_i the mean of 1/|x - r_i| over the point's own element or face.
//
// Here the charges are a sparse matrix C (points x dofs, built on the host
// at assembly), the point-to-point sum is a direct N-body kernel in FP64,
// and apply_selfgrav subtracts C^T S C X from a K_eff product. The direct
// sum costs O(points^2) per column; the paper applies S by FMM.
//
// The self distances are integrated in polar coordinates about the foot of
// the barycentre in each face plane, in closed form (element:
// int_K dx/|x - r| = sum_F (h_F / 2) int_F dA / |y - r| over the cones from
// r; face: the point lies in the plane, h = 0).
#include <algorithm>
#include <cmath>
#include <vector>

#include "kernels.h"
#include "nm_internal.h"

namespace nm {

namespace {

struct V3 {
    double x, y, z;
};
inline V3 sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 add(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 mul(V3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
inline double norm(V3 a) { return std::sqrt(dot(a, a)); }

// int over triangle (a, b, c) of dA / |y - p|: polar coordinates about the
// foot f of p in the triangle's plane (p at height h), one signed
// sub-triangle (f, edge) per edge. For an edge at distance d from f, with
// s the coordinate along the edge from the perpendicular's foot and
// R(s) = sqrt(d^2 + h^2 + s^2) the distance from p, the radial integral
// int_0^{r(phi)} rho d rho / sqrt(rho^2 + h^2) = sqrt(r^2 + h^2) - h with
// r = d / cos(phi), tan(phi) = s / d, integrates in phi to
//   F(s) = d asinh(s / sqrt(d^2 + h^2)) + h atan(h s / (d R(s))) - h atan(s / d),
// and the sub-triangle contributes F(s_B) - F(s_A).
double tri_inv_dist(V3 a, V3 b, V3 c, V3 p) {
    V3 n = cross(sub(b, a), sub(c, a));
    n = mul(n, 1.0 / norm(n));
    const double hs = dot(sub(p, a), n);
    const double h = std::fabs(hs);
    const V3 f = sub(p, mul(n, hs));
    const V3 P[3] = {a, b, c};
    double total = 0.0;
    for (int e = 0; e < 3; ++e) {
        const V3 A = sub(P[e], f), B = sub(P[(e + 1) % 3], f);
        const V3 ed = sub(B, A);
        const double len = norm(ed);
        const V3 t = mul(ed, 1.0 / len);
        const double sA = dot(A, t), sB = dot(B, t);
        const V3 cr = cross(A, B);
        const double d = norm(cr) / len;
        if (d <= 1e-14 * len) continue;   // f on the edge line: empty sub-triangle
        const double sgn = dot(cr, n) >= 0 ? 1.0 : -1.0;
        const double q = std::sqrt(d * d + h * h);
        auto F = [&](double sv) {
            const double R = std::sqrt(q * q + sv * sv);
            return d * std::asinh(sv / q) + h * std::atan(h * sv / (d * R)) - h * std::atan(sv / d);
        };
        total += sgn * (F(sB) - F(sA));
    }
    return total;
}

__global__ void csr_spmm_kernel(int64_t nrows, const int64_t* __restrict__ rowptr, const int* __restrict__ col,
                                const double* __restrict__ val, const double* __restrict__ X, int64_t ldx, double* Y,
                                int64_t ldy, int b, double alpha, double beta) {
    // one warp per row; lane c handles columns c and c + 32
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= nrows) return;
    double s0 = 0.0, s1 = 0.0;
    for (int64_t e = rowptr[row]; e < rowptr[row + 1]; ++e) {
        const double v = val[e];
        const double* x = X + (int64_t)col[e] * ldx;
        if (lane < b) s0 += v * x[lane];
        if (lane + 32 < b) s1 += v * x[lane + 32];
    }
    double* y = Y + row * ldy;
    if (lane < b) y[lane] = alpha * s0 + (beta == 0.0 ? 0.0 : beta * y[lane]);
    if (lane + 32 < b) y[lane + 32] = alpha * s1 + (beta == 0.0 ? 0.0 : beta * y[lane + 32]);
}

constexpr int kTile = 128;   // targets per CTA and sources per shared-memory stage

// 1/sqrt(r2) to double accuracy: the float estimate refined by one Newton
// step for f(y) = 1/y^2 - r2, y <- y (3 - r2 y^2) / 2, which squares its
// relative error (rsqrtf's ~1e-7 becomes ~2e-14). Four FP64 operations
// instead of a full double-precision reciprocal square root.
__device__ __forceinline__ double inv_dist(double r2) {
    const double y = (double)rsqrtf((float)r2);
    return y * fma(-0.5 * r2, y * y, 1.5);
}

// Phi[i, c] = G sum_{j != i} Q[j, c] / |r_i - r_j| + G inv_R[i] Q[i, c].
// One thread per target and group of NC columns (blockIdx.y): one 1/r per
// pair serves NC products, so the FP64 pipe spends ~10 of its 10 + NC
// operations per pair on the distance. The sources pass through shared
// memory kTile at a time. With split > 1 (small point sets, to fill the
// machine) CTA z sums the sources of its range [z chunk, (z + 1) chunk) into
// part[z] and nbody_reduce_kernel adds the ranges in order.
template <int NC>
__global__ void __launch_bounds__(kTile) nbody_kernel(int64_t np, const double* __restrict__ pts,
                                                     const double* __restrict__ inv_R, double G,
                                                     const double* __restrict__ Q, int b, double* Phi,
                                                     int64_t chunk, double* part) {
    __shared__ double sx[kTile], sy[kTile], sz[kTile];
    __shared__ __align__(16) double sq[kTile][NC];
    const int c0 = blockIdx.y * NC;
    const int nc = b - c0 < NC ? b - c0 : NC;
    const int64_t i = blockIdx.x * (int64_t)kTile + threadIdx.x;
    const int64_t jb = blockIdx.z * chunk;
    const int64_t je = jb + chunk < np ? jb + chunk : np;
    double xi = 0, yi = 0, zi = 0;
    if (i < np) {
        xi = pts[3 * i];
        yi = pts[3 * i + 1];
        zi = pts[3 * i + 2];
    }
    double acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = 0.0;
    for (int64_t j0 = jb; j0 < je; j0 += kTile) {
        const int64_t j = j0 + threadIdx.x;
        const bool in = j < je;
        sx[threadIdx.x] = in ? pts[3 * j] : 0.0;
        sy[threadIdx.x] = in ? pts[3 * j + 1] : 0.0;
        sz[threadIdx.x] = in ? pts[3 * j + 2] : 0.0;
#pragma unroll
        for (int c = 0; c < NC; ++c) sq[threadIdx.x][c] = (in && c < nc) ? Q[j * b + c0 + c] : 0.0;
        __syncthreads();
        const int cnt = je - j0 < kTile ? (int)(je - j0) : kTile;
        const int64_t self = i - j0;   // the target's own slot in this stage, if any
        for (int k = 0; k < cnt; ++k) {
            const double dx = sx[k] - xi, dy = sy[k] - yi, dz = sz[k] - zi;
            const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
            const double w = (k == self) ? 0.0 : inv_dist(r2);
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[c] = fma(sq[k][c], w, acc[c]);
        }
        __syncthreads();
    }
    if (i >= np) return;
    if (part) {
        double* o = part + ((int64_t)blockIdx.z * np + i) * b + c0;
#pragma unroll
        for (int c = 0; c < NC; ++c)
            if (c < nc) o[c] = acc[c];
        return;
    }
    const double d = inv_R[i];
#pragma unroll
    for (int c = 0; c < NC; ++c)
        if (c < nc) Phi[i * b + c0 + c] = G * fma(d, Q[i * b + c0 + c], acc[c]);
}

// Phi = G (sum over the source ranges of part + inv_R Q), ranges in order.
__global__ void nbody_reduce_kernel(int64_t np, int b, int split, const double* __restrict__ part,
                                    const double* __restrict__ inv_R, double G, const double* __restrict__ Q,
                                    double* Phi) {
    const int64_t total = np * b;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int z = 0; z < split; ++z) acc += part[z * total + t];
        Phi[t] = G * fma(inv_R[t / b], Q[t], acc);
    }
}

// CTAs the n-body launch aims for: several waves of 128-thread CTAs on 152 SMs.
constexpr int64_t kNbodyCtas = 2048;
constexpr int kMaxSplit = 32;

int nbody_cols(int b) { return b <= 8 ? 8 : (b <= 16 ? 16 : 32); }

// Source ranges for an n-body sum over np points with b columns.
int nbody_split(int64_t np, int b) {
    const int64_t tiles = (np + kTile - 1) / kTile;
    const int64_t groups = (b + nbody_cols(b) - 1) / nbody_cols(b);
    int64_t sp = (kNbodyCtas + tiles * groups - 1) / (tiles * groups);
    if (sp > kMaxSplit) sp = kMaxSplit;
    if (sp > tiles) sp = tiles;
    if (sp < 1) sp = 1;
    // equal ranges of whole tiles; drop the ones left empty by the rounding
    const int64_t per = (tiles + sp - 1) / sp;
    return (int)((tiles + per - 1) / per);
}

template <int NC>
void launch_nbody(int64_t np, const double* pts, const double* inv_R, double G, const double* Q, int b, double* Phi,
                  double* part, cudaStream_t s) {
    const int split = nbody_split(np, b);
    const int64_t tiles = (np + kTile - 1) / kTile;
    const int64_t chunk = ((tiles + split - 1) / split) * kTile;
    dim3 grid((unsigned)tiles, (unsigned)((b + NC - 1) / NC), (unsigned)split);
    nbody_kernel<NC><<<grid, kTile, 0, s>>>(np, pts, inv_R, G, Q, b, Phi, chunk, split > 1 ? part : nullptr);
    if (split > 1) {
        count_launch();
        const int64_t total = np * b;
        const int blocks = (int)std::min<int64_t>((total + 255) / 256, 4096);
        nbody_reduce_kernel<<<blocks, 256, 0, s>>>(np, b, split, part, inv_R, G, Q, Phi);
    }
}

struct Entry {
    int64_t row;
    int32_t col;
    double val;
};

int upload_csr(std::vector<Entry>& ent, int64_t nrows, DevBuf& rp, DevBuf& cl, DevBuf& vl) {
    std::sort(ent.begin(), ent.end(), [](const Entry& a, const Entry& b) {
        return a.row != b.row ? a.row < b.row : a.col < b.col;
    });
    std::vector<int64_t> h_rp(nrows + 1, 0);
    std::vector<int32_t> h_c;
    std::vector<double> h_v;
    for (size_t k = 0; k < ent.size(); ++k) {
        if (!h_c.empty() && k > 0 && ent[k].row == ent[k - 1].row && ent[k].col == ent[k - 1].col) {
            h_v.back() += ent[k].val;
            continue;
        }
        h_rp[ent[k].row + 1] += 1;
        h_c.push_back(ent[k].col);
        h_v.push_back(ent[k].val);
    }
    for (int64_t r = 0; r < nrows; ++r) h_rp[r + 1] += h_rp[r];
    NM_TRY(rp.alloc(h_rp.size() * sizeof(int64_t)));
    NM_TRY(cl.alloc(std::max<size_t>(h_c.size(), 1) * sizeof(int32_t)));
    NM_TRY(vl.alloc(std::max<size_t>(h_v.size(), 1) * sizeof(double)));
    NM_CUDA(cudaMemcpy(rp.p, h_rp.data(), h_rp.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    if (!h_c.empty()) {
        NM_CUDA(cudaMemcpy(cl.p, h_c.data(), h_c.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
        NM_CUDA(cudaMemcpy(vl.p, h_v.data(), h_v.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    return NM_OK;
}

}  // namespace

// Charge points, self distances and the charge matrices of the problem.
// tet10: P2 ids per tet (vertices, then edges (0,1), (0,2), (0,3), (1,2),
// (1,3), (2,3)); usol / uflu: internal u-node of the solid / fluid copy of
// each P2 node (-1 if none).
// Host part: the points (3 per point), their inverse self distances and the
// entries (point, dof, value) of C, duplicates not yet summed.
void self_gravity_host(const double* xyz, const int32_t* tet, const int64_t* tet10, const uint8_t* region,
                       const double* rho, int64_t nt, const int32_t* usol, const int32_t* uflu,
                       std::vector<double>& pts, std::vector<double>& invR, std::vector<int64_t>& erow,
                       std::vector<int32_t>& ecol, std::vector<double>& eval) {
    static const int kE[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
    static const int kF[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
    auto vtx = [&](int64_t v) { return V3{xyz[3 * v], xyz[3 * v + 1], xyz[3 * v + 2]}; };
    std::vector<Entry> ent;
    pts.clear();
    invR.clear();
    ent.reserve(18 * nt);
    // elements
    for (int64_t t = 0; t < nt; ++t) {
        V3 v[4];
        for (int a = 0; a < 4; ++a) v[a] = vtx(tet[4 * t + a]);
        const V3 e1 = sub(v[1], v[0]), e2 = sub(v[2], v[0]), e3 = sub(v[3], v[0]);
        const double det = dot(e1, cross(e2, e3));
        const double vol = std::fabs(det) / 6.0;
        // gradients of the barycentric coordinates: rows of the inverse Jacobian
        V3 g[4];
        g[1] = mul(cross(e2, e3), 1.0 / det);
        g[2] = mul(cross(e3, e1), 1.0 / det);
        g[3] = mul(cross(e1, e2), 1.0 / det);
        g[0] = mul(add(add(g[1], g[2]), g[3]), -1.0);
        const int64_t row = (int64_t)(pts.size() / 3);
        const int32_t* un = region[t] ? uflu : usol;
        for (int e = 0; e < 6; ++e) {
            const V3 w = mul(add(g[kE[e][0]], g[kE[e][1]]), rho[t] * vol);
            const int32_t node = un[tet10[10 * t + 4 + e]];
            ent.push_back({row, 3 * node + 0, w.x});
            ent.push_back({row, 3 * node + 1, w.y});
            ent.push_back({row, 3 * node + 2, w.z});
        }
        const V3 r = mul(add(add(v[0], v[1]), add(v[2], v[3])), 0.25);
        double s = 0.0;
        for (int f = 0; f < 4; ++f) {
            const V3 a = v[kF[f][0]], b = v[kF[f][1]], c = v[kF[f][2]];
            V3 nrm = cross(sub(b, a), sub(c, a));
            const double hF = std::fabs(dot(sub(r, a), nrm)) / norm(nrm);
            s += 0.5 * hF * tri_inv_dist(a, b, c, r);
        }
        pts.insert(pts.end(), {r.x, r.y, r.z});
        invR.push_back(s / vol);
    }
    // faces: sort the 4 nt faces by their vertex triple
    struct Face {
        int32_t k[3];
        int64_t t;
        int f;
    };
    std::vector<Face> faces(4 * nt);
    for (int64_t t = 0; t < nt; ++t)
        for (int f = 0; f < 4; ++f) {
            int32_t k[3] = {tet[4 * t + kF[f][0]], tet[4 * t + kF[f][1]], tet[4 * t + kF[f][2]]};
            std::sort(k, k + 3);
            faces[4 * t + f] = {{k[0], k[1], k[2]}, t, f};
        }
    std::sort(faces.begin(), faces.end(), [](const Face& a, const Face& b) {
        for (int i = 0; i < 3; ++i)
            if (a.k[i] != b.k[i]) return a.k[i] < b.k[i];
        return a.t < b.t;
    });
    // local edge index of vertex pair (i, j) in a tet
    auto local_edge = [&](int i, int j) {
        for (int e = 0; e < 6; ++e)
            if ((kE[e][0] == i && kE[e][1] == j) || (kE[e][0] == j && kE[e][1] == i)) return e;
        return -1;
    };
    // a charged face: edge nodes of the face in tet t (local face f) with
    // weight coef * nu * |E| / 3 on the given copy; nu points away from t's
    // opposite vertex
    auto face_geom = [&](int64_t t, int f, V3* nu, double* area, V3* bary, V3 tri[3]) {
        for (int i = 0; i < 3; ++i) tri[i] = vtx(tet[4 * t + kF[f][i]]);
        V3 nn = cross(sub(tri[1], tri[0]), sub(tri[2], tri[0]));
        const double len = norm(nn);
        nn = mul(nn, 1.0 / len);
        const V3 opp = vtx(tet[4 * t + f]);
        if (dot(sub(opp, tri[0]), nn) > 0) nn = mul(nn, -1.0);
        *nu = nn;
        *area = 0.5 * len;
        *bary = mul(add(add(tri[0], tri[1]), tri[2]), 1.0 / 3.0);
    };
    auto add_face_charges = [&](int64_t row, int64_t t, int f, V3 nu, double w, const int32_t* copy) {
        for (int a = 0; a < 3; ++a)
            for (int c = a + 1; c < 3; ++c) {
                const int e = local_edge(kF[f][a], kF[f][c]);
                const int32_t node = copy[tet10[10 * t + 4 + e]];
                ent.push_back({row, 3 * node + 0, w * nu.x});
                ent.push_back({row, 3 * node + 1, w * nu.y});
                ent.push_back({row, 3 * node + 2, w * nu.z});
            }
    };
    auto face_selfdist = [&](V3 tri[3], V3 bary, double area) {
        return tri_inv_dist(tri[0], tri[1], tri[2], bary) / area;
    };
    size_t i = 0;
    while (i < faces.size()) {
        size_t j = i + 1;
        while (j < faces.size() && faces[j].k[0] == faces[i].k[0] && faces[j].k[1] == faces[i].k[1] &&
               faces[j].k[2] == faces[i].k[2])
            ++j;
        if (j - i == 1) {
            // outer boundary: -rho_inside (nu . u), nu outward
            const Face& F = faces[i];
            V3 nu, bary, tri[3];
            double area;
            face_geom(F.t, F.f, &nu, &area, &bary, tri);
            const int64_t row = (int64_t)(pts.size() / 3);
            add_face_charges(row, F.t, F.f, nu, -rho[F.t] * area / 3.0, region[F.t] ? uflu : usol);
            pts.insert(pts.end(), {bary.x, bary.y, bary.z});
            invR.push_back(face_selfdist(tri, bary, area));
        } else if (j - i == 2 && region[faces[i].t] == region[faces[i + 1].t] &&
                   rho[faces[i].t] != rho[faces[i + 1].t]) {
            // density jump inside a region: (rho_+ - rho_-) (nu . u), nu from - to +
            const Face& Mi = faces[i];
            const Face& Pl = faces[i + 1];
            V3 nu, bary, tri[3];
            double area;
            face_geom(Mi.t, Mi.f, &nu, &area, &bary, tri);
            const int64_t row = (int64_t)(pts.size() / 3);
            add_face_charges(row, Mi.t, Mi.f, nu, (rho[Pl.t] - rho[Mi.t]) * area / 3.0, region[Mi.t] ? uflu : usol);
            pts.insert(pts.end(), {bary.x, bary.y, bary.z});
            invR.push_back(face_selfdist(tri, bary, area));
        } else if (j - i == 2 && region[faces[i].t] != region[faces[i + 1].t]) {
            // fluid-solid: rho_f (nu . u^f) - rho_s (nu . u^s), nu from solid to fluid
            const Face& S = region[faces[i].t] == 0 ? faces[i] : faces[i + 1];
            const Face& Fl = region[faces[i].t] == 0 ? faces[i + 1] : faces[i];
            V3 nu, bary, tri[3];
            double area;
            face_geom(S.t, S.f, &nu, &area, &bary, tri);
            const int64_t row = (int64_t)(pts.size() / 3);
            add_face_charges(row, S.t, S.f, nu, -rho[S.t] * area / 3.0, usol);
            add_face_charges(row, S.t, S.f, nu, rho[Fl.t] * area / 3.0, uflu);
            pts.insert(pts.end(), {bary.x, bary.y, bary.z});
            invR.push_back(face_selfdist(tri, bary, area));
        }
        i = j;
    }
    erow.resize(ent.size());
    ecol.resize(ent.size());
    eval.resize(ent.size());
    for (size_t k = 0; k < ent.size(); ++k) {
        erow[k] = ent[k].row;
        ecol[k] = ent[k].col;
        eval[k] = ent[k].val;
    }
}

int build_self_gravity(nm_problem* P, const double* xyz, const int32_t* tet, const int64_t* tet10,
                       const uint8_t* region, const double* rho, int64_t nt, const int32_t* usol,
                       const int32_t* uflu, double G) {
    const int64_t n = P->info.n;
    std::vector<double> pts, invR, ev;
    std::vector<int64_t> er;
    std::vector<int32_t> ec;
    self_gravity_host(xyz, tet, tet10, region, rho, nt, usol, uflu, pts, invR, er, ec, ev);
    std::vector<Entry> ent(er.size());
    for (size_t k = 0; k < er.size(); ++k) ent[k] = {er[k], ec[k], ev[k]};
    const int64_t np = (int64_t)invR.size();
    SelfGravity& SG = P->sg;
    SG.np = np;
    SG.G = G;
    NM_TRY(SG.pts.alloc(pts.size() * sizeof(double)));
    NM_TRY(SG.invR.alloc(invR.size() * sizeof(double)));
    NM_CUDA(cudaMemcpy(SG.pts.p, pts.data(), pts.size() * sizeof(double), cudaMemcpyHostToDevice));
    NM_CUDA(cudaMemcpy(SG.invR.p, invR.data(), invR.size() * sizeof(double), cudaMemcpyHostToDevice));
    std::vector<Entry> tr(ent.size());
    for (size_t k = 0; k < ent.size(); ++k) tr[k] = {ent[k].col, (int32_t)ent[k].row, ent[k].val};
    NM_TRY(upload_csr(ent, np, SG.c_rp, SG.c_col, SG.c_val));
    NM_TRY(upload_csr(tr, n, SG.t_rp, SG.t_col, SG.t_val));
    NM_TRY(SG.q.alloc((size_t)np * 64 * sizeof(double)));
    NM_TRY(SG.phi.alloc((size_t)np * 64 * sizeof(double)));
    // partial sums of the split n-body launches, for the widest need over b
    size_t part = 0;
    for (int b = 1; b <= 64; ++b) {
        const int sp = nbody_split(np, b);
        if (sp > 1) part = std::max(part, (size_t)sp * np * b);
    }
    if (part) NM_TRY(SG.part.alloc(part * sizeof(double)));
    SG.on = 1;
    return NM_OK;
}

// W -= C^T S C X for a block of b <= 64 columns (X, W row-major FP64).
int apply_selfgrav(nm_problem* P, const double* X, int64_t ldx, double* W, int64_t ldw, int b, cudaStream_t s) {
    SelfGravity& SG = P->sg;
    if (!SG.on) return NM_OK;
    if (b < 1 || b > 64) return fail(NM_EINVAL, "self-gravitation takes blocks of 1..64 columns");
    const int64_t n = P->info.n;
    const int per = 256 / 32;
    csr_spmm_kernel<<<(unsigned)((SG.np + per - 1) / per), 256, 0, s>>>(
        SG.np, SG.c_rp.as<int64_t>(), SG.c_col.as<int>(), SG.c_val.as<double>(), X, ldx, SG.q.as<double>(), b, b,
        1.0, 0.0);
    count_launch();
    NM_CUDA(cudaGetLastError());
    // the narrowest column group that holds the block (wider blocks: groups of 32)
    const double *pts = SG.pts.as<double>(), *invR = SG.invR.as<double>(), *q = SG.q.as<double>();
    double *phi = SG.phi.as<double>(), *part = SG.part.as<double>();
    if (nbody_cols(b) == 8)
        launch_nbody<8>(SG.np, pts, invR, SG.G, q, b, phi, part, s);
    else if (nbody_cols(b) == 16)
        launch_nbody<16>(SG.np, pts, invR, SG.G, q, b, phi, part, s);
    else
        launch_nbody<32>(SG.np, pts, invR, SG.G, q, b, phi, part, s);
    count_launch();
    NM_CUDA(cudaGetLastError());
    csr_spmm_kernel<<<(unsigned)((n + per - 1) / per), 256, 0, s>>>(
        n, SG.t_rp.as<int64_t>(), SG.t_col.as<int>(), SG.t_val.as<double>(), SG.phi.as<double>(), b, W, ldw, b, -1.0,
        1.0);
    count_launch();
    NM_CUDA(cudaGetLastError());
    return NM_OK;
}

}  // namespace nm
