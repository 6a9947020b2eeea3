// Host-side, once-per-topology rest-state precompute in FP64 (not on the timed path).
//
//  * D_m^{-1} per triangle (Appendix B, F = D_s D_m^{-1}); D_m is the rest edge pair
//    [X_j - X_i, X_k - X_i] written in an orthonormal frame of the rest triangle,
//    taken here as the upper-triangular factor of the rest Gram matrix.
//  * rest areas W (Sec. 2.1.3, E_i = W_i Psi(F_i)),
//  * cotangent weights divided by twice the mixed Voronoi area and the rest
//    Laplacian vectors delta_g (Sec. 2.1.2, Eq. BendingDiscretizedPotential),
//  * lumped masses (Sec. 2.1.1), rest volume V0 (Sec. 2.1.2),
//  * L = sum_i w_i G_i^T G_i as a sparse symmetric matrix (Eq. fullyDeveloped_g),
//    with the area term (w = C * W), the optional material term (k_mat_hess * W,
//    Sec. 2.1.1), the bending term (w = k_bend * A_i) and the volume term (G = I).
#include <math.h>

#include <algorithm>
#include <cstring>
#include <utility>

#include "npfem_internal.h"

namespace npfem {
namespace {

struct V3 {
    double x, y, z;
};
inline V3 sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 add(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 scale(V3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
inline double norm(V3 a) { return sqrt(dot(a, a)); }

// Sparse symmetric accumulator with short rows.
struct RowAccum {
    std::vector<std::vector<std::pair<int, double>>> rows;
    explicit RowAccum(int n) : rows(n) {}
    void add(int i, int j, double v)
    {
        for (auto& e : rows[i])
            if (e.first == j) {
                e.second += v;
                return;
            }
        rows[i].push_back({j, v});
    }
};

}  // namespace

int build_host_topo(const npfem_mesh* mesh, const npfem_material* mat, int equal_mass, HostTopo* o, std::string* err)
{
    const int n = mesh->n_verts, nt = mesh->n_tris;
    if (n < 4 || nt < 4 || n > 65535) {
        *err = "mesh needs 4..65535 vertices and >= 4 triangles";
        return NPFEM_ERR_INVALID_ARG;
    }
    // --- topology check: every directed edge once, every reverse edge present
    std::vector<unsigned long long> dir;
    dir.reserve(3 * (size_t)nt);
    for (int t = 0; t < nt; ++t)
        for (int a = 0; a < 3; ++a) {
            int i = mesh->tris[3 * t + a], j = mesh->tris[3 * t + (a + 1) % 3];
            if (i < 0 || i >= n || j < 0 || j >= n || i == j) {
                *err = "triangle " + std::to_string(t) + " has an invalid or repeated vertex index";
                return NPFEM_ERR_BAD_MESH;
            }
            dir.push_back(((unsigned long long)i << 32) | (unsigned)j);
        }
    std::sort(dir.begin(), dir.end());
    for (size_t q = 1; q < dir.size(); ++q)
        if (dir[q] == dir[q - 1]) {
            *err = "directed edge used twice: faces are not consistently oriented or the mesh is non-manifold";
            return NPFEM_ERR_BAD_MESH;
        }
    for (unsigned long long e : dir) {
        unsigned long long r = ((e & 0xffffffffull) << 32) | (e >> 32);
        if (!std::binary_search(dir.begin(), dir.end(), r)) {
            *err = "mesh has a boundary edge (not closed) or inconsistent orientation";
            return NPFEM_ERR_BAD_MESH;
        }
    }
    std::vector<char> used(n, 0);
    for (int q = 0; q < 3 * nt; ++q) used[mesh->tris[q]] = 1;
    for (int i = 0; i < n; ++i)
        if (!used[i]) {
            *err = "vertex " + std::to_string(i) + " belongs to no triangle";
            return NPFEM_ERR_BAD_MESH;
        }

    o->n = n;
    o->nt = nt;
    o->tri.assign(mesh->tris, mesh->tris + 3 * nt);
    auto X = [&](int i) { return V3{mesh->rest_xyz[3 * i], mesh->rest_xyz[3 * i + 1], mesh->rest_xyz[3 * i + 2]}; };

    // --- one-ring adjacency (sorted neighbour lists)
    std::vector<std::vector<int>> nb(n);
    for (unsigned long long e : dir) nb[e >> 32].push_back((int)(e & 0xffffffffull));
    for (auto& r : nb) std::sort(r.begin(), r.end());
    auto slot = [&](int i, int j) { return (int)(std::lower_bound(nb[i].begin(), nb[i].end(), j) - nb[i].begin()); };

    o->dminv.assign(4 * (size_t)nt, 0.0);
    o->W.assign(nt, 0.0);
    o->avor.assign(n, 0.0);
    std::vector<double> bary(n, 0.0);
    std::vector<std::vector<double>> cot(n);
    for (int i = 0; i < n; ++i) cot[i].assign(nb[i].size(), 0.0);
    std::vector<V3> nrest(n, V3{0, 0, 0});
    double A0 = 0.0, V0 = 0.0;

    for (int t = 0; t < nt; ++t) {
        const int vi[3] = {mesh->tris[3 * t], mesh->tris[3 * t + 1], mesh->tris[3 * t + 2]};
        V3 P[3] = {X(vi[0]), X(vi[1]), X(vi[2])};
        V3 e1 = sub(P[1], P[0]), e2 = sub(P[2], P[0]);
        V3 cr = cross(e1, e2);
        double twoA = norm(cr);
        double g11 = dot(e1, e1), g12 = dot(e1, e2);
        if (!(twoA > 1e-14 * g11) || !(g11 > 0.0)) {
            *err = "rest triangle " + std::to_string(t) + " is degenerate";
            return NPFEM_ERR_BAD_MESH;
        }
        // D_m = [[l1, g12/l1], [0, 2A/l1]] (upper-triangular Gram factor)
        double l1 = sqrt(g11), a = l1, b = g12 / l1, c = twoA / l1;
        double* Di = &o->dminv[4 * (size_t)t];
        Di[0] = 1.0 / a;
        Di[1] = -b / (a * c);
        Di[2] = 0.0;
        Di[3] = 1.0 / c;
        double area = 0.5 * twoA;
        o->W[t] = area;
        A0 += area;
        V0 += dot(P[0], cr) / 6.0;
        for (int q = 0; q < 3; ++q) {
            bary[vi[q]] += area / 3.0;
            nrest[vi[q]] = add(nrest[vi[q]], scale(cr, 0.5));
        }
        // corner cotangents (corner q is opposite the edge of the other two corners)
        double ct[3];
        for (int q = 0; q < 3; ++q) {
            V3 u = sub(P[(q + 1) % 3], P[q]), w = sub(P[(q + 2) % 3], P[q]);
            ct[q] = dot(u, w) / norm(cross(u, w));
            int p1 = vi[(q + 1) % 3], p2 = vi[(q + 2) % 3];
            cot[p1][slot(p1, p2)] += ct[q];
            cot[p2][slot(p2, p1)] += ct[q];
        }
        // mixed Voronoi area (Meyer et al. 2003)
        int obt = -1;
        for (int q = 0; q < 3; ++q)
            if (ct[q] < 0.0) obt = q;
        for (int q = 0; q < 3; ++q) {
            if (obt >= 0) {
                o->avor[vi[q]] += (q == obt) ? 0.5 * area : 0.25 * area;
            } else {
                int q1 = (q + 1) % 3, q2 = (q + 2) % 3;
                V3 to1 = sub(P[q1], P[q]), to2 = sub(P[q2], P[q]);
                // edge q-q1 is opposite corner q2, edge q-q2 opposite corner q1
                o->avor[vi[q]] += 0.125 * (dot(to1, to1) * ct[q2] + dot(to2, to2) * ct[q1]);
            }
        }
    }
    if (!(V0 > 0.0)) {
        *err = "rest volume is not positive: faces must be counter-clockwise seen from outside";
        return NPFEM_ERR_BAD_MESH;
    }
    o->A0 = A0;
    o->V0 = V0;

    // --- one-ring CSR with c_ij = (cot a + cot b) / (2 A_i), delta_g, mean edge length
    o->ring_ptr.assign(n + 1, 0);
    o->ring_idx.clear();
    o->ring_c.clear();
    o->dg_norm.assign(n, 0.0);
    o->csum.assign(n, 0.0);
    o->nsign.assign(n, 1.0);
    o->bend_w.assign(n, 0.0);
    double lsum = 0.0;
    long ecount = 0;
    for (int i = 0; i < n; ++i) {
        o->ring_ptr[i] = (int)o->ring_idx.size();
        V3 dg{0, 0, 0};
        double cs = 0.0;
        for (size_t q = 0; q < nb[i].size(); ++q) {
            int j = nb[i][q];
            double cij = cot[i][q] / (2.0 * o->avor[i]);
            o->ring_idx.push_back(j);
            o->ring_c.push_back(cij);
            dg = add(dg, scale(sub(X(j), X(i)), cij));
            cs += cij;
            if (j > i) {
                lsum += norm(sub(X(j), X(i)));
                ecount++;
            }
        }
        o->dg_norm[i] = norm(dg);
        o->csum[i] = cs;
        o->nsign[i] = dot(dg, nrest[i]) >= 0.0 ? 1.0 : -1.0;
        o->bend_w[i] = mat->k_bend * o->avor[i];
    }
    o->ring_ptr[n] = (int)o->ring_idx.size();
    o->lbar = lsum / (double)ecount;
    // transposed weights: the bending gradient is gathered per vertex, which needs
    // the weight each neighbour's ring gives to this vertex
    o->ring_ct.assign(o->ring_idx.size(), 0.0);
    for (int i = 0; i < n; ++i)
        for (int q = o->ring_ptr[i]; q < o->ring_ptr[i + 1]; ++q) {
            const int j = o->ring_idx[q];
            for (int p = o->ring_ptr[j]; p < o->ring_ptr[j + 1]; ++p)
                if (o->ring_idx[p] == i) o->ring_ct[q] = o->ring_c[p];
        }
    // vertex -> (triangle, corner) incidence, for gathering per-triangle gradients
    o->inc_ptr.assign(n + 1, 0);
    for (int q = 0; q < 3 * nt; ++q) o->inc_ptr[mesh->tris[q] + 1]++;
    for (int i = 0; i < n; ++i) o->inc_ptr[i + 1] += o->inc_ptr[i];
    o->inc_idx.assign(3 * (size_t)nt, 0);
    {
        std::vector<int> fillp(o->inc_ptr.begin(), o->inc_ptr.end() - 1);
        for (int t = 0; t < nt; ++t)
            for (int a = 0; a < 3; ++a) o->inc_idx[fillp[mesh->tris[3 * t + a]]++] = (t << 2) | a;
    }

    // --- lumped masses
    o->mtotal = mat->density * V0;
    o->mass.assign(n, 0.0);
    for (int i = 0; i < n; ++i) o->mass[i] = equal_mass ? o->mtotal / n : o->mtotal * bary[i] / A0;
    // rest positions about the rest centre of mass (frame of the learned warm start)
    {
        V3 cm{0, 0, 0};
        double mt = 0.0;
        for (int i = 0; i < n; ++i) {
            cm = add(cm, scale(X(i), o->mass[i]));
            mt += o->mass[i];
        }
        cm = scale(cm, 1.0 / mt);
        o->rest_c.assign(3 * (size_t)n, 0.0);
        for (int i = 0; i < n; ++i) {
            const V3 r = sub(X(i), cm);
            o->rest_c[i] = r.x;
            o->rest_c[n + i] = r.y;
            o->rest_c[2 * n + i] = r.z;
        }
    }

    // --- L = sum_i w_i G_i^T G_i (sparse)
    RowAccum L(n);
    const double wA = mat->C + mat->k_mat_hess;
    for (int t = 0; t < nt; ++t) {
        const int vi[3] = {mesh->tris[3 * t], mesh->tris[3 * t + 1], mesh->tris[3 * t + 2]};
        const double* Di = &o->dminv[4 * (size_t)t];
        for (int col = 0; col < 2; ++col) {
            // column col of F = (x_j - x_i) Di[0][col] + (x_k - x_i) Di[1][col]
            double gj = Di[col], gk = Di[2 + col];
            double g[3] = {-(gj + gk), gj, gk};
            for (int p = 0; p < 3; ++p)
                for (int q = 0; q < 3; ++q) L.add(vi[p], vi[q], wA * o->W[t] * g[p] * g[q]);
        }
    }
    for (int i = 0; i < n; ++i) {
        double w = o->bend_w[i];
        int b = o->ring_ptr[i], e = o->ring_ptr[i + 1];
        for (int p = b; p <= e; ++p) {
            int vp = (p == e) ? i : o->ring_idx[p];
            double gp = (p == e) ? -o->csum[i] : o->ring_c[p];
            for (int q = b; q <= e; ++q) {
                int vq = (q == e) ? i : o->ring_idx[q];
                double gq = (q == e) ? -o->csum[i] : o->ring_c[q];
                L.add(vp, vq, w * gp * gq);
            }
        }
        L.add(i, i, mat->k_vol);
    }
    o->L_ptr.assign(n + 1, 0);
    o->L_idx.clear();
    o->L_val.clear();
    for (int i = 0; i < n; ++i) {
        auto& r = L.rows[i];
        std::sort(r.begin(), r.end());
        o->L_ptr[i] = (int)o->L_idx.size();
        for (auto& e : r) {
            o->L_idx.push_back(e.first);
            o->L_val.push_back(e.second);
        }
    }
    o->L_ptr[n] = (int)o->L_idx.size();
    return NPFEM_OK;
}

}  // namespace npfem
