// Host-side setup of the operator-split step: mesh adjacency and geometry,
// model validation, the time window tau and the fixed-point face tables
// (Parallel STEPS §2.1), and the Morton or reverse Cuthill-McKee order of tets.
//
// Floating-point notes: this file is compiled without contraction
// (-ffp-contract=off). Volumes, areas, barycentre distances, face rates,
// tau and the thresholds are evaluated in the fixed operation order written
// here, so any independent implementation that writes the same formulas in
// the same order gets the same bits.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <limits>
#include <numeric>

#include "steps_internal.h"

namespace steps {

namespace {

// Local face f of a tet is the triangle opposite its local vertex f.
constexpr int kFaceVerts[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};

inline void sub3(const double *a, const double *b, double *o) {
    o[0] = a[0] - b[0];
    o[1] = a[1] - b[1];
    o[2] = a[2] - b[2];
}

inline void cross3(const double *u, const double *w, double *o) {
    o[0] = u[1] * w[2] - u[2] * w[1];
    o[1] = u[2] * w[0] - u[0] * w[2];
    o[2] = u[0] * w[1] - u[1] * w[0];
}

// |det(b-a, c-a, d-a)| / 6
double volume(const double *a, const double *b, const double *c, const double *d) {
    double u[3], v[3], w[3], x[3];
    sub3(b, a, u);
    sub3(c, a, v);
    sub3(d, a, w);
    cross3(v, w, x);
    double det = u[0] * x[0] + u[1] * x[1] + u[2] * x[2];
    return std::fabs(det) / 6.0;
}

// |(q-p) x (r-p)| / 2
double area(const double *p, const double *q, const double *r) {
    double u[3], w[3], x[3];
    sub3(q, p, u);
    sub3(r, p, w);
    cross3(u, w, x);
    return 0.5 * std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
}

struct FaceKey {
    std::array<int32_t, 3> v;
    int32_t tet;
    int32_t face;
};

uint64_t spread3(uint64_t x) {  // 21 bits -> every third bit of 63
    x &= 0x1fffff;
    x = (x | x << 32) & 0x001f00000000ffffULL;
    x = (x | x << 16) & 0x001f0000ff0000ffULL;
    x = (x | x << 8) & 0x100f00f00f00f00fULL;
    x = (x | x << 4) & 0x10c30c30c30c30c3ULL;
    x = (x | x << 2) & 0x1249249249249249ULL;
    return x;
}

}  // namespace

int build_mesh(const double *verts, int64_t nv, const int32_t *tets, int64_t nt, HostMesh &m) {
    if (!verts || !tets || nv < 4 || nt < 1 || nt > (int64_t)INT32_MAX / 4) {
        set_error("steps_mesh_create: need nv >= 4, 1 <= nt < 2^29 and non-NULL arrays");
        return STEPS_ERR_ARG;
    }
    m.nv = nv;
    m.nt = nt;
    m.verts.assign(verts, verts + 3 * nv);
    m.tets.assign(tets, tets + 4 * nt);
    for (int64_t i = 0; i < 4 * nt; ++i) {
        if (tets[i] < 0 || tets[i] >= nv) {
            set_error("steps_mesh_create: vertex index out of range in tet " + std::to_string(i / 4));
            return STEPS_ERR_MESH;
        }
    }
    // adjacency: sort faces by their sorted vertex triple; equal triples are neighbours
    std::vector<FaceKey> faces((size_t)(4 * nt));
    for (int64_t i = 0; i < nt; ++i) {
        for (int f = 0; f < 4; ++f) {
            FaceKey &k = faces[(size_t)(4 * i + f)];
            for (int j = 0; j < 3; ++j) k.v[j] = tets[4 * i + kFaceVerts[f][j]];
            std::sort(k.v.begin(), k.v.end());
            k.tet = (int32_t)i;
            k.face = f;
        }
    }
    std::sort(faces.begin(), faces.end(), [](const FaceKey &a, const FaceKey &b) {
        if (a.v != b.v) return a.v < b.v;
        if (a.tet != b.tet) return a.tet < b.tet;
        return a.face < b.face;
    });
    m.nbr.assign((size_t)(4 * nt), -1);
    for (size_t j = 0; j < faces.size();) {
        size_t e = j + 1;
        while (e < faces.size() && faces[e].v == faces[j].v) ++e;
        if (e - j > 2) {
            set_error("steps_mesh_create: a face is shared by more than two tets (tet " +
                      std::to_string(faces[j].tet) + ")");
            return STEPS_ERR_MESH;
        }
        if (e - j == 2) {
            if (faces[j].tet == faces[j + 1].tet) {
                set_error("steps_mesh_create: tet " + std::to_string(faces[j].tet) + " repeats a vertex");
                return STEPS_ERR_MESH;
            }
            m.nbr[(size_t)(4 * faces[j].tet + faces[j].face)] = faces[j + 1].tet;
            m.nbr[(size_t)(4 * faces[j + 1].tet + faces[j + 1].face)] = faces[j].tet;
        }
        j = e;
    }
    // volumes and barycentres
    m.vol.resize((size_t)nt);
    m.bary.resize((size_t)(3 * nt));
    for (int64_t i = 0; i < nt; ++i) {
        const double *p[4];
        for (int j = 0; j < 4; ++j) p[j] = verts + 3 * (int64_t)tets[4 * i + j];
        m.vol[(size_t)i] = volume(p[0], p[1], p[2], p[3]);
        if (!(m.vol[(size_t)i] > 0.0)) {
            set_error("steps_mesh_create: tet " + std::to_string(i) + " has zero volume");
            return STEPS_ERR_MESH;
        }
        for (int c = 0; c < 3; ++c)
            m.bary[(size_t)(3 * i + c)] = (((p[0][c] + p[1][c]) + p[2][c]) + p[3][c]) * 0.25;
    }
    // geometric face rates g = A / (V d), d = barycentre distance
    m.g.assign((size_t)(4 * nt), 0.0);
    for (int64_t i = 0; i < nt; ++i) {
        const double *p[4];
        for (int j = 0; j < 4; ++j) p[j] = verts + 3 * (int64_t)tets[4 * i + j];
        const double *ci = &m.bary[(size_t)(3 * i)];
        for (int f = 0; f < 4; ++f) {
            int32_t j = m.nbr[(size_t)(4 * i + f)];
            if (j < 0) continue;
            double a = area(p[kFaceVerts[f][0]], p[kFaceVerts[f][1]], p[kFaceVerts[f][2]]);
            const double *cj = &m.bary[(size_t)(3 * j)];
            double dx = cj[0] - ci[0], dy = cj[1] - ci[1], dz = cj[2] - ci[2];
            double d = std::sqrt(dx * dx + dy * dy + dz * dz);
            m.g[(size_t)(4 * i + f)] = a / (m.vol[(size_t)i] * d);
        }
    }
    return STEPS_OK;
}

int build_model(int32_t S, const double *D, int32_t R, const int32_t *lhs, const int32_t *rhs,
                const double *k, HostModel &m) {
    if (S < 1 || S > kMaxSpecies || R < 0 || R > kMaxReac || !D || (R > 0 && (!lhs || !rhs || !k))) {
        set_error("steps_model_create: need 1 <= n_species <= 32, 0 <= n_reac <= 32, non-NULL arrays");
        return STEPS_ERR_ARG;
    }
    m.S = S;
    m.R = R;
    m.D.assign(D, D + S);
    m.lhs.clear();
    m.rhs.clear();
    m.k.clear();
    if (R > 0) {
        m.lhs.assign(lhs, lhs + (size_t)R * S);
        m.rhs.assign(rhs, rhs + (size_t)R * S);
        m.k.assign(k, k + R);
    }
    std::memset(&m.dev, 0, sizeof(m.dev));
    m.dev.S = S;
    m.dev.R = R;
    for (int s = 0; s < S; ++s) {
        if (!(D[s] >= 0.0) || !std::isfinite(D[s])) {
            set_error("steps_model_create: diffusion constant of species " + std::to_string(s) + " is invalid");
            return STEPS_ERR_MODEL;
        }
        if (D[s] > 0.0) m.dev.diffusive |= 1u << s;
    }
    for (int r = 0; r < R; ++r) {
        ReacDesc &d = m.dev.reac[r];
        if (!(k[r] >= 0.0) || !std::isfinite(k[r])) {
            set_error("steps_model_create: rate constant of reaction " + std::to_string(r) + " is invalid");
            return STEPS_ERR_MODEL;
        }
        int order = 0, ra = -1, rb = -1, nchg = 0;
        for (int s = 0; s < S; ++s) {
            int l = lhs[(size_t)r * S + s], q = rhs[(size_t)r * S + s];
            if (l < 0 || q < 0 || l > 2 || q > 100) {
                set_error("steps_model_create: bad stoichiometry in reaction " + std::to_string(r));
                return STEPS_ERR_MODEL;
            }
            for (int c = 0; c < l; ++c) {
                if (ra < 0) ra = s; else rb = s;
                ++order;
            }
            int delta = q - l;
            if (delta != 0) {
                if (nchg >= kMaxChanges) {
                    set_error("steps_model_create: reaction " + std::to_string(r) + " changes more than 6 species");
                    return STEPS_ERR_MODEL;
                }
                d.chg_s[nchg] = (int8_t)s;
                d.chg_d[nchg] = (int8_t)delta;
                ++nchg;
            }
        }
        if (order > 2) {
            set_error("steps_model_create: reaction " + std::to_string(r) + " has order > 2");
            return STEPS_ERR_MODEL;
        }
        d.k = (float)k[r];
        d.need = (ra >= 0 ? 1u << ra : 0u) | (rb >= 0 ? 1u << rb : 0u);
        d.nchg = nchg;
        d.type = order == 0 ? kOrder0 : order == 1 ? kOrder1 : (ra == rb ? kDimer : kOrder2);
        d.ia = ra >= 0 ? ra : S;
        d.ib = rb >= 0 ? rb : S;
        d.sub = d.type == kDimer ? 1 : 0;
        if (d.type == kOrder0) m.dev.order0 |= 1u << r;
    }
    return STEPS_OK;
}

namespace {

// Reverse Cuthill-McKee order of the face-adjacency graph. Components are
// taken in the order of their lowest-degree (then lowest-index) tet; each
// is searched breadth-first from a pseudo-peripheral tet (the lowest-degree
// tet of the last level of a search from that tet), visiting a tet's
// unvisited neighbours by increasing degree, then index; the whole sequence
// is reversed. Face neighbours end up few positions apart (a narrow band).
void rcm_order(const HostMesh &mesh, int64_t nt, std::vector<int32_t> &perm) {
    std::vector<int8_t> deg((size_t)nt, 0);
    for (int64_t i = 0; i < nt; ++i)
        for (int f = 0; f < 4; ++f) deg[(size_t)i] += mesh.nbr[(size_t)(4 * i + f)] >= 0 ? 1 : 0;
    auto before = [&](int32_t a, int32_t b) { return deg[(size_t)a] < deg[(size_t)b] || (deg[(size_t)a] == deg[(size_t)b] && a < b); };
    std::vector<int32_t> by_deg((size_t)nt);
    std::iota(by_deg.begin(), by_deg.end(), 0);
    std::stable_sort(by_deg.begin(), by_deg.end(), [&](int32_t a, int32_t b) { return deg[(size_t)a] < deg[(size_t)b]; });
    std::vector<int32_t> stamp((size_t)nt, -1), frontier, next, last;
    int32_t cur_stamp = 0;
    auto far_tet = [&](int32_t s) {
        ++cur_stamp;
        stamp[(size_t)s] = cur_stamp;
        frontier.assign(1, s);
        while (!frontier.empty()) {
            last = frontier;
            next.clear();
            for (int32_t u : frontier)
                for (int f = 0; f < 4; ++f) {
                    const int32_t v = mesh.nbr[(size_t)(4 * (int64_t)u + f)];
                    if (v >= 0 && stamp[(size_t)v] != cur_stamp) {
                        stamp[(size_t)v] = cur_stamp;
                        next.push_back(v);
                    }
                }
            frontier.swap(next);
        }
        int32_t best = last[0];
        for (int32_t v : last)
            if (before(v, best)) best = v;
        return best;
    };
    std::vector<uint8_t> seen((size_t)nt, 0);
    std::vector<int32_t> order;
    order.reserve((size_t)nt);
    for (int32_t s0 : by_deg) {
        if (seen[(size_t)s0]) continue;
        const int32_t s = far_tet(s0);
        size_t head = order.size();
        order.push_back(s);
        seen[(size_t)s] = 1;
        while (head < order.size()) {
            const int32_t u = order[head++];
            int32_t nb[4];
            int n = 0;
            for (int f = 0; f < 4; ++f) {
                const int32_t v = mesh.nbr[(size_t)(4 * (int64_t)u + f)];
                if (v >= 0 && !seen[(size_t)v]) {
                    seen[(size_t)v] = 1;
                    nb[n++] = v;
                }
            }
            std::sort(nb, nb + n, before);
            order.insert(order.end(), nb, nb + n);
        }
    }
    std::reverse(order.begin(), order.end());
    perm.swap(order);
}

}  // namespace

void build_tables(const HostMesh &mesh, const HostModel &model, int reorder, Tables &t) {
    const int64_t nt = mesh.nt;
    // tau = 1 / max_{S,tet} D_S G_tet over diffusive species (§2.1); the max of
    // the products is the product of the maxima because rounding is monotone.
    t.dmax = 0.0;
    for (double d : model.D) t.dmax = std::max(t.dmax, d);
    std::vector<double> cumg((size_t)(4 * nt));
    t.gmax = 0.0;
    for (int64_t i = 0; i < nt; ++i) {
        double c = 0.0;
        for (int f = 0; f < 4; ++f) {
            c = c + mesh.g[(size_t)(4 * i + f)];
            cumg[(size_t)(4 * i + f)] = c;
        }
        if (c > t.gmax) t.gmax = c;
    }
    t.tau = (t.dmax > 0.0 && t.gmax > 0.0) ? 1.0 / (t.dmax * t.gmax) : std::numeric_limits<double>::infinity();

    // device order
    t.perm.resize((size_t)nt);
    std::iota(t.perm.begin(), t.perm.end(), 0);
    if (reorder == STEPS_REORDER_MORTON && nt > 1) {
        double lo[3], hi[3];
        for (int c = 0; c < 3; ++c) {
            lo[c] = std::numeric_limits<double>::infinity();
            hi[c] = -lo[c];
        }
        for (int64_t i = 0; i < nt; ++i)
            for (int c = 0; c < 3; ++c) {
                lo[c] = std::min(lo[c], mesh.bary[(size_t)(3 * i + c)]);
                hi[c] = std::max(hi[c], mesh.bary[(size_t)(3 * i + c)]);
            }
        double span = std::max({hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2], 1e-300});
        std::vector<uint64_t> code((size_t)nt);
        for (int64_t i = 0; i < nt; ++i) {
            uint64_t q[3];
            for (int c = 0; c < 3; ++c) {
                double x = (mesh.bary[(size_t)(3 * i + c)] - lo[c]) / span * 2097151.0;
                q[c] = (uint64_t)std::min(2097151.0, std::max(0.0, x));
            }
            code[(size_t)i] = spread3(q[0]) | spread3(q[1]) << 1 | spread3(q[2]) << 2;
        }
        std::stable_sort(t.perm.begin(), t.perm.end(),
                         [&](int32_t a, int32_t b) { return code[(size_t)a] < code[(size_t)b]; });
    } else if (reorder == STEPS_REORDER_RCM && nt > 1) {
        rcm_order(mesh, nt, t.perm);
    }
    t.inv_perm.resize((size_t)nt);
    for (int64_t d = 0; d < nt; ++d) t.inv_perm[(size_t)t.perm[(size_t)d]] = (int32_t)d;

    // fixed-point cumulative thresholds: EULER A_{i,f} = floor(2^31 tau Dmax cumg_{i,f});
    // EXP the face shares floor(2^31 cumg_{i,f} / G_i) (the leave probability is per
    // species and tet, exp_leave_table)
    double pt = std::isfinite(t.tau) ? t.tau * t.dmax : 0.0;
    t.nbr_dev.resize((size_t)(4 * nt));
    t.thr_dev.resize((size_t)(4 * nt));
    t.inv_nav_dev.resize((size_t)nt);
    t.G_dev.resize((size_t)nt);
    for (int64_t d = 0; d < nt; ++d) {
        int64_t i = t.perm[(size_t)d];
        const double G = cumg[(size_t)(4 * i + 3)];
        t.G_dev[(size_t)d] = G;
        for (int f = 0; f < 4; ++f) {
            int32_t j = mesh.nbr[(size_t)(4 * i + f)];
            t.nbr_dev[(size_t)(4 * d + f)] = j < 0 ? -1 : t.inv_perm[(size_t)j];
            double fl;
            if (model.leave_exp) fl = G > 0.0 ? std::floor((cumg[(size_t)(4 * i + f)] / G) * 2147483648.0) : 0.0;
            else fl = std::floor((pt * cumg[(size_t)(4 * i + f)]) * 2147483648.0);
            fl = std::min(2147483648.0, std::max(0.0, fl));
            t.thr_dev[(size_t)(4 * d + f)] = (uint32_t)fl;
        }
        double nav = kAvogadro * (mesh.vol[(size_t)i] * 1000.0);
        t.inv_nav_dev[(size_t)d] = (float)(1.0 / nav);
    }
}

void exp_leave_table(const HostModel &model, const Tables &t, double tau_k, size_t Tpad, std::vector<uint32_t> &out) {
    const size_t T = t.G_dev.size();
    out.assign((size_t)model.S * Tpad, 0u);
    if (!std::isfinite(t.tau)) return;
    for (int s = 0; s < model.S; ++s) {
        const double D = model.D[(size_t)s];
        if (!(D > 0.0)) continue;
        for (size_t d = 0; d < T; ++d) {
            const double x = (tau_k * D) * t.G_dev[d];
            double fl = std::floor((1.0 - std::exp(-x)) * 2147483648.0);
            fl = std::min(2147483648.0, std::max(0.0, fl));
            out[(size_t)s * Tpad + d] = (uint32_t)fl;
        }
    }
}

// R_S = floor(2^31 (D_S / Dmax) (tau_k / tau)), clamped to [0, 2^31].
uint32_t species_scale(const HostModel &model, const Tables &t, int s, double tau_k) {
    if (!(model.D[(size_t)s] > 0.0) || !std::isfinite(t.tau)) return 0;
    double x = ((model.D[(size_t)s] / t.dmax) * (tau_k / t.tau)) * 2147483648.0;
    double fl = std::floor(x);
    fl = std::min(2147483648.0, std::max(0.0, fl));
    return (uint32_t)fl;
}

}  // namespace steps
