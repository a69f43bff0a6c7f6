// Host-side set-up of sim_create: per-tet constants, lumped masses, surface extraction, objects, rest-pose
// exclusion (Sec. 5.1) and the vertex -> (tet, corner) lists of the segmented scatter.
#include <algorithm>
#include <array>
#include <cmath>
#include <numeric>
#include <unordered_map>

#include "geometry.cuh"
#include "sim.h"

namespace pncg {

namespace {

struct Face { int a, b, c; };

long long cell_id(long long i, long long j, long long k)
{
    const long long B = 1 << 20;
    return ((i + B) << 42) | ((j + B) << 21) | (k + B);
}

// pairs of one object closer than r at the rest positions X (brute-force distance on grid candidates)
void rest_exclusions(const std::vector<double> &X, HostMesh &m, double r)
{
    if (r <= 0 || m.nf == 0) return;
    double Ls = 0;
    for (int e = 0; e < m.ne; ++e) {
        const double *a = &X[3 * m.edge[4 * e]], *b = &X[3 * m.edge[4 * e + 1]];
        Ls += std::sqrt((a[0] - b[0]) * (a[0] - b[0]) + (a[1] - b[1]) * (a[1] - b[1]) + (a[2] - b[2]) * (a[2] - b[2]));
    }
    const double cell = std::max(Ls / std::max(m.ne, 1), r);
    auto box = [&](const int *v, int n, double infl, long long lo[3], long long hi[3]) {
        for (int a = 0; a < 3; ++a) {
            double l = 1e300, h = -1e300;
            for (int k = 0; k < n; ++k) { l = std::min(l, X[3 * v[k] + a]); h = std::max(h, X[3 * v[k] + a]); }
            lo[a] = (long long)std::floor((l - infl) / cell);
            hi[a] = (long long)std::floor((h + infl) / cell);
        }
    };
    auto P = [&](int v) { return v3<double>{X[3 * v], X[3 * v + 1], X[3 * v + 2]}; };
    std::vector<unsigned long long> keys;
    // point-triangle
    std::unordered_map<long long, std::vector<int>> grid;
    for (int f = 0; f < m.nf; ++f) {
        long long lo[3], hi[3];
        box(&m.tri[4 * f], 3, r, lo, hi);
        for (long long i = lo[0]; i <= hi[0]; ++i)
            for (long long j = lo[1]; j <= hi[1]; ++j)
                for (long long k = lo[2]; k <= hi[2]; ++k) grid[cell_id(i, j, k)].push_back(f);
    }
    for (int a = 0; a < m.ns; ++a) {
        const int v = m.svert[a];
        auto it = grid.find(cell_id((long long)std::floor(X[3 * v] / cell), (long long)std::floor(X[3 * v + 1] / cell),
                                    (long long)std::floor(X[3 * v + 2] / cell)));
        if (it == grid.end()) continue;
        for (int f : it->second) {
            const int *t = &m.tri[4 * f];
            if (t[0] == v || t[1] == v || t[2] == v || t[3] != m.obj[v]) continue;
            double c[4];
            v3<double> tt;
            double d = pt_coeffs<double>(P(v) - P(t[0]), P(t[1]) - P(t[0]), P(t[2]) - P(t[0]), c, tt);
            if (d < r) keys.push_back(((unsigned long long)a << 31) | (unsigned long long)f);
        }
    }
    // edge-edge
    grid.clear();
    for (int e = 0; e < m.ne; ++e) {
        long long lo[3], hi[3];
        box(&m.edge[4 * e], 2, r, lo, hi);
        for (long long i = lo[0]; i <= hi[0]; ++i)
            for (long long j = lo[1]; j <= hi[1]; ++j)
                for (long long k = lo[2]; k <= hi[2]; ++k) grid[cell_id(i, j, k)].push_back(e);
    }
    std::vector<int> seen(m.ne, -1);
    for (int a = 0; a < m.ne; ++a) {
        const int *ea = &m.edge[4 * a];
        long long lo[3], hi[3];
        box(ea, 2, 0.0, lo, hi);
        for (long long i = lo[0]; i <= hi[0]; ++i)
            for (long long j = lo[1]; j <= hi[1]; ++j)
                for (long long k = lo[2]; k <= hi[2]; ++k) {
                    auto it = grid.find(cell_id(i, j, k));
                    if (it == grid.end()) continue;
                    for (int b : it->second) {
                        if (b <= a || seen[b] == a) continue;
                        seen[b] = a;
                        const int *eb = &m.edge[4 * b];
                        if (eb[0] == ea[0] || eb[0] == ea[1] || eb[1] == ea[0] || eb[1] == ea[1] || eb[2] != ea[2]) continue;
                        double c[4];
                        v3<double> tt;
                        double d = ee_coeffs<double>(P(ea[0]) - P(eb[0]), P(ea[1]) - P(eb[0]), P(eb[1]) - P(eb[0]), c, tt);
                        if (d < r) keys.push_back((1ull << 62) | ((unsigned long long)a << 31) | (unsigned long long)b);
                    }
                }
    }
    std::sort(keys.begin(), keys.end());
    m.excl = keys;
}

} // namespace

sim_status build_host_mesh(const sim_mesh *mesh, const sim_material *mat, double dt, double dhat, double kappa,
                           const sim_options &opt, HostMesh &m, std::string &err)
{
    if (!mesh || !mat) { err = "mesh and material are required"; return SIM_ERR_INVALID_ARG; }
    if (mesh->n_verts <= 0 || mesh->n_tets <= 0 || !mesh->rest_x || !mesh->tets) { err = "empty mesh"; return SIM_ERR_INVALID_ARG; }
    if (!(dt > 0) || !(dhat > 0) || !(kappa >= 0) || !std::isfinite(dt) || !std::isfinite(dhat) || !std::isfinite(kappa)) {
        err = "dt and dhat must be positive and kappa non-negative";
        return SIM_ERR_INVALID_ARG;
    }
    if (!(mat->density > 0) || !(mat->poisson > -1.0 && mat->poisson < 0.5) || !(mat->youngs >= 0)) {
        err = "density must be positive, poisson in (-1, 0.5), youngs >= 0";
        return SIM_ERR_INVALID_ARG;
    }
    if (opt.iters <= 0 || opt.beta < 0 || opt.beta > 1 || opt.pnorm < 0 || opt.pnorm > 1 || opt.precision < 0 ||
        opt.precision > 1 || opt.scatter < 0 || opt.scatter > 3 || opt.persistent < 0 || opt.persistent > 2 ||
        opt.split_objects < 0 || opt.split_objects > 2 || opt.block_shape < -1 || opt.block_shape > 4) {
        err = "invalid options";
        return SIM_ERR_INVALID_ARG;
    }
    if (mat->model < SIM_MAT_NH || mat->model > SIM_MAT_ARAP) { err = "unknown material model"; return SIM_ERR_INVALID_ARG; }
    const int nv = mesh->n_verts, nt = mesh->n_tets;
    m.nv = nv; m.nt = nt; m.h = dt; m.dhat = dhat; m.kappa = kappa; m.opt = opt;
    m.model = mat->model;
    const double nu = mat->poisson;
    const double Eb = mat->youngs_per_tet ? 1.0 : mat->youngs;
    m.nu = nu;
    m.mu = Eb / (2.0 * (1.0 + nu));
    m.lam = Eb * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    const double *X = mesh->rest_x;
    m.X.assign(X, X + 3 * (size_t)nv);
    m.x0.assign(mesh->x0 ? mesh->x0 : X, (mesh->x0 ? mesh->x0 : X) + 3 * (size_t)nv);
    m.v0.assign(3 * (size_t)nv, 0.0);
    if (mesh->v0) std::copy(mesh->v0, mesh->v0 + 3 * (size_t)nv, m.v0.begin());
    for (double q : m.x0) if (!std::isfinite(q)) { err = "non-finite initial position"; return SIM_ERR_INVALID_ARG; }
    for (double q : m.v0) if (!std::isfinite(q)) { err = "non-finite initial velocity"; return SIM_ERR_INVALID_ARG; }
    m.tet.assign(mesh->tets, mesh->tets + 4 * (size_t)nt);
    m.Dm.assign(9 * (size_t)nt, 0.0);
    m.hv.assign(nt, 0.0);
    m.mass.assign(nv, 0.0);
    if (mat->youngs_per_tet) {
        m.escale.assign(mat->youngs_per_tet, mat->youngs_per_tet + nt);
        for (double e : m.escale) if (!(e >= 0) || !std::isfinite(e)) { err = "invalid per-tet Young's modulus"; return SIM_ERR_INVALID_ARG; }
    }
    for (int e = 0; e < nt; ++e) {
        const int *v = &m.tet[4 * e];
        for (int i = 0; i < 4; ++i)
            if (v[i] < 0 || v[i] >= nv) { err = "tet " + std::to_string(e) + " has a vertex index out of range"; return SIM_ERR_INVALID_ARG; }
        double A[3][3];
        for (int c = 0; c < 3; ++c)
            for (int a = 0; a < 3; ++a) A[a][c] = X[3 * v[c + 1] + a] - X[3 * v[0] + a];
        const double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                           A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
        if (!(det > 0)) { err = "tet " + std::to_string(e) + " has non-positive rest volume"; return SIM_ERR_INVALID_ARG; }
        // inverse by cofactors: Inv[r][c] = cof(A)[c][r] / det
        double I[3][3];
        I[0][0] = (A[1][1] * A[2][2] - A[1][2] * A[2][1]) / det;
        I[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / det;
        I[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / det;
        I[1][0] = (A[1][2] * A[2][0] - A[1][0] * A[2][2]) / det;
        I[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / det;
        I[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / det;
        I[2][0] = (A[1][0] * A[2][1] - A[1][1] * A[2][0]) / det;
        I[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / det;
        I[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / det;
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) m.Dm[(size_t)(3 * r + c) * nt + e] = I[r][c];
        const double vol = det / 6.0;
        m.hv[e] = dt * dt * vol;
        for (int i = 0; i < 4; ++i) m.mass[v[i]] += mat->density * vol / 4.0;
    }
    // objects: connected components over tet vertices
    m.obj.resize(nv);
    std::iota(m.obj.begin(), m.obj.end(), 0);
    auto root = [&](int a) { while (m.obj[a] != a) { m.obj[a] = m.obj[m.obj[a]]; a = m.obj[a]; } return a; };
    for (int e = 0; e < nt; ++e)
        for (int k = 1; k < 4; ++k) {
            int a = root(m.tet[4 * e]), b = root(m.tet[4 * e + k]);
            if (a != b) m.obj[std::max(a, b)] = std::min(a, b);
        }
    for (int i = 0; i < nv; ++i) m.obj[i] = root(i);
    // surface: faces that belong to exactly one tet
    std::vector<std::array<int, 3>> faces;
    faces.reserve(4 * (size_t)nt);
    static const int fv[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
    for (int e = 0; e < nt; ++e)
        for (int f = 0; f < 4; ++f) {
            std::array<int, 3> q = {m.tet[4 * e + fv[f][0]], m.tet[4 * e + fv[f][1]], m.tet[4 * e + fv[f][2]]};
            std::sort(q.begin(), q.end());
            faces.push_back(q);
        }
    std::sort(faces.begin(), faces.end());
    std::vector<std::array<int, 3>> surf;
    for (size_t i = 0; i < faces.size();) {
        size_t j = i + 1;
        while (j < faces.size() && faces[j] == faces[i]) ++j;
        if (j - i == 1) surf.push_back(faces[i]);
        i = j;
    }
    m.nf = (int)surf.size();
    m.tri.resize(4 * (size_t)m.nf);
    std::vector<std::array<int, 2>> edges;
    std::vector<char> on(nv, 0);
    for (int f = 0; f < m.nf; ++f) {
        const auto &q = surf[f];
        m.tri[4 * f] = q[0]; m.tri[4 * f + 1] = q[1]; m.tri[4 * f + 2] = q[2]; m.tri[4 * f + 3] = m.obj[q[0]];
        edges.push_back({q[0], q[1]}); edges.push_back({q[1], q[2]}); edges.push_back({q[0], q[2]});
        on[q[0]] = on[q[1]] = on[q[2]] = 1;
    }
    std::sort(edges.begin(), edges.end());
    edges.erase(std::unique(edges.begin(), edges.end()), edges.end());
    m.ne = (int)edges.size();
    m.edge.resize(4 * (size_t)m.ne);
    for (int e = 0; e < m.ne; ++e) {
        m.edge[4 * e] = edges[e][0]; m.edge[4 * e + 1] = edges[e][1]; m.edge[4 * e + 2] = m.obj[edges[e][0]]; m.edge[4 * e + 3] = 0;
    }
    m.svert.clear();
    for (int i = 0; i < nv; ++i) if (on[i]) m.svert.push_back(i);
    m.ns = (int)m.svert.size();
    // kinematic vertices
    m.fix_slot.assign(nv, -1);
    m.nfix = 0;
    if (mesh->fixed)
        for (int i = 0; i < nv; ++i) if (mesh->fixed[i]) m.fix_slot[i] = m.nfix++;
    // rest-pose exclusion of same-object pairs
    rest_exclusions(std::vector<double>(X, X + 3 * (size_t)nv), m, opt.excl_factor * dhat);
    {
        double Ls = 0;
        for (int e = 0; e < m.ne; ++e) {
            const double *a = &X[3 * (size_t)m.edge[4 * e]], *b = &X[3 * (size_t)m.edge[4 * e + 1]];
            Ls += std::sqrt((a[0] - b[0]) * (a[0] - b[0]) + (a[1] - b[1]) * (a[1] - b[1]) + (a[2] - b[2]) * (a[2] - b[2]));
        }
        m.edge_mean = m.ne > 0 ? Ls / m.ne : 0.0;
    }
    // vertex -> (tet, corner) CSR in tet order
    m.v2c_off.assign(nv + 1, 0);
    for (int q = 0; q < 4 * nt; ++q) m.v2c_off[m.tet[q] + 1]++;
    for (int i = 0; i < nv; ++i) m.v2c_off[i + 1] += m.v2c_off[i];
    m.v2c.assign(4 * (size_t)nt, 0);
    std::vector<int> cur(m.v2c_off.begin(), m.v2c_off.end() - 1);
    for (int q = 0; q < 4 * nt; ++q) m.v2c[cur[m.tet[q]]++] = q;
    // batching: scenes (validated: ids 0 .. S-1, non-decreasing over the vertices, every id present, each tet
    // inside one scene, tets ordered by scene)
    m.nseg = 1;
    m.vscene.clear();
    if (mesh->scene_of_vert) {
        const int32_t *sc = mesh->scene_of_vert;
        if (sc[0] != 0) { err = "scene_of_vert must start at 0"; return SIM_ERR_INVALID_ARG; }
        for (int i = 1; i < nv; ++i)
            if (sc[i] != sc[i - 1] && sc[i] != sc[i - 1] + 1) {
                err = "scene_of_vert must be non-decreasing in steps of 1 (vertex " + std::to_string(i) + ")";
                return SIM_ERR_INVALID_ARG;
            }
        m.nseg = sc[nv - 1] + 1;
        if (m.nseg > MAX_SCENES) { err = "at most " + std::to_string(MAX_SCENES) + " scenes"; return SIM_ERR_INVALID_ARG; }
        int prev = 0;
        for (int e = 0; e < nt; ++e) {
            const int *v = &m.tet[4 * (size_t)e];
            const int s0 = sc[v[0]];
            if (sc[v[1]] != s0 || sc[v[2]] != s0 || sc[v[3]] != s0) {
                err = "tet " + std::to_string(e) + " spans two scenes";
                return SIM_ERR_INVALID_ARG;
            }
            if (s0 < prev) { err = "tets must be ordered by scene (tet " + std::to_string(e) + ")"; return SIM_ERR_INVALID_ARG; }
            prev = s0;
        }
        if (m.nseg > 1) m.vscene.assign(sc, sc + nv);
    }
    // collision / non-collision parts: two groups per object (vscene keeps the objects)
    m.nobj = m.nseg;
    if (opt.split_objects == 2) {
        if (m.vscene.empty()) m.vscene.assign(nv, 0);
        m.nseg = 2 * m.nobj;
        if (m.nseg > MAX_SCENES) { err = "at most " + std::to_string(MAX_SCENES / 2) + " objects with parts"; return SIM_ERR_INVALID_ARG; }
    }
    // block-scatter tables
    const int nchunk = (nt + SCATTER_CHUNK - 1) / SCATTER_CHUNK;
    m.cv_off.assign(nchunk + 1, 0);
    m.cv.clear();
    m.tloc.assign(4 * (size_t)nt, 0);
    std::vector<int> ids;
    for (int c = 0; c < nchunk; ++c) {
        const int e0 = c * SCATTER_CHUNK, e1 = std::min(nt, e0 + SCATTER_CHUNK);
        ids.assign(m.tet.begin() + 4 * (size_t)e0, m.tet.begin() + 4 * (size_t)e1);
        std::sort(ids.begin(), ids.end());
        ids.erase(std::unique(ids.begin(), ids.end()), ids.end());
        for (int q = 4 * e0; q < 4 * e1; ++q)
            m.tloc[q] = (unsigned short)(std::lower_bound(ids.begin(), ids.end(), m.tet[q]) - ids.begin());
        m.cv.insert(m.cv.end(), ids.begin(), ids.end());
        m.cv_off[c + 1] = (int)m.cv.size();
    }
    // colouring scatter: first-fit greedy colouring of the tets (the colours a vertex's tets already have are a
    // bit mask per vertex), then the tets grouped by colour
    m.color_off.clear();
    m.color_tets.clear();
    if (opt.scatter == SIM_SCATTER_COLOR) {
        if (m.nseg > 1) { err = "the colouring scatter runs one kernel per phase: not with batched scenes"; return SIM_ERR_INVALID_ARG; }
        std::vector<unsigned long long> used(nv, 0ull);
        std::vector<int> col(nt);
        int ncol = 0;
        for (int e = 0; e < nt; ++e) {
            const int *v = &m.tet[4 * (size_t)e];
            const unsigned long long busy = used[v[0]] | used[v[1]] | used[v[2]] | used[v[3]];
            if (busy == ~0ull) { err = "the colouring scatter needs more than 64 colours"; return SIM_ERR_INVALID_ARG; }
            int c = 0;
            while (busy >> c & 1ull) ++c;
            col[e] = c;
            ncol = std::max(ncol, c + 1);
            for (int i = 0; i < 4; ++i) used[v[i]] |= 1ull << c;
        }
        m.color_off.assign(ncol + 1, 0);
        for (int e = 0; e < nt; ++e) ++m.color_off[col[e] + 1];
        for (int c = 0; c < ncol; ++c) m.color_off[c + 1] += m.color_off[c];
        std::vector<int> pos(m.color_off.begin(), m.color_off.end() - 1);
        m.color_tets.resize(nt);
        for (int e = 0; e < nt; ++e) m.color_tets[pos[col[e]]++] = e;
    }
    return SIM_OK;
}

} // namespace pncg
