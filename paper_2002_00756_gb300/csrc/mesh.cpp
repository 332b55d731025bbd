// Host-side construction of the cubed-sphere hierarchy and the Helmholtz coefficients.
//
// Mesh: equiangular gnomonic cubed sphere C_n as used for the paper's experiments
// (Maynard, Melvin & Mueller, arXiv 2002.00756, Sec. 5.1: C192 / C1152 meshes; Sec. 4:
// horizontal partition, contiguous vertical columns).  Coarse levels are C_{n/2}, ...
// (Sec. 3.6: horizontal-only coarsening; the equiangular C_{n/2} cell is exactly the
// union of 2x2 C_n cells).  Coefficients follow Eq. helmholtz_operator in strong,
// volume-normalised, lowest-order form (see mgsolve.h).
//
// Geometry here is computed independently of any other implementation:
//   * cell areas from the closed-form area of an equiangular gnomonic cell,
//     A = R^2 [F(x2,y2) - F(x1,y2) - F(x2,y1) + F(x1,y1)], F(x,y) = atan(x y / sqrt(1+x^2+y^2)),
//     x = tan(xi), y = tan(eta) (Rancic, Purser & Mesinger 1996);
//   * neighbours by stepping three quarters of a cell across each edge in the panel's
//     (extended) gnomonic coordinates, projecting to the sphere and locating the cell
//     that contains the point with the inverse gnomonic map;
//   * edge lengths and centre distances as great-circle arcs.
#include "mesh.h"

#include <cmath>
#include <cstdio>

namespace mg {
namespace {

struct V3 {
    double x, y, z;
};

V3 cube_point(int p, double a, double b) {
    switch (p) {
        case 0: return {1.0, a, b};
        case 1: return {-a, 1.0, b};
        case 2: return {-1.0, -a, b};
        case 3: return {a, -1.0, b};
        case 4: return {-b, a, 1.0};
        default: return {b, a, -1.0};
    }
}

V3 unit(V3 v) {
    const double r = std::sqrt(v.x * v.x + v.y * v.y + v.z * v.z);
    return {v.x / r, v.y / r, v.z / r};
}

V3 sphere(int p, double xi, double eta) { return unit(cube_point(p, std::tan(xi), std::tan(eta))); }

double arc(V3 u, V3 v) {
    const double cx = u.y * v.z - u.z * v.y, cy = u.z * v.x - u.x * v.z, cz = u.x * v.y - u.y * v.x;
    return std::atan2(std::sqrt(cx * cx + cy * cy + cz * cz), u.x * v.x + u.y * v.y + u.z * v.z);
}

// Inverse gnomonic map: panel and (tan xi, tan eta) of a point on the sphere.
void locate(V3 v, int& p, double& a, double& b) {
    const double ax = std::fabs(v.x), ay = std::fabs(v.y), az = std::fabs(v.z);
    if (ax >= ay && ax >= az) {
        if (v.x > 0) { p = 0; a = v.y / v.x; b = v.z / v.x; }
        else         { p = 2; a = v.y / v.x; b = -v.z / v.x; }
    } else if (ay >= az) {
        if (v.y > 0) { p = 1; a = -v.x / v.y; b = v.z / v.y; }
        else         { p = 3; a = -v.x / v.y; b = -v.z / v.y; }
    } else {
        if (v.z > 0) { p = 4; a = v.y / v.z; b = -v.x / v.z; }
        else         { p = 5; a = -v.y / v.z; b = -v.x / v.z; }
    }
}

double gnomonic_F(double x, double y) { return std::atan(x * y / std::sqrt(1.0 + x * x + y * y)); }

}  // namespace

std::string build_hgeom(int n, double radius, HGeom& g) {
    if (n < 1) return "n must be >= 1";
    const double PI = 3.14159265358979323846;
    const double d = 0.5 * PI / n, q = 0.25 * PI;
    const int ncol = 6 * n * n;
    g.n = n;
    g.ncol = ncol;
    g.area.assign(ncol, 0.0);
    g.sinlat.assign(ncol, 0.0);
    g.nbr.assign(4 * ncol, -1);
    g.nbr_side.assign(4 * ncol, -1);
    g.edge_len.assign(4 * ncol, 0.0);
    g.cdist.assign(4 * ncol, 0.0);
    std::vector<V3> centre(ncol);
    const double R2 = radius * radius;
    // side offsets in (i, j) for E, W, N, S
    const int di[4] = {1, -1, 0, 0}, dj[4] = {0, 0, 1, -1};
    for (int c = 0; c < ncol; ++c) {
        const int p = c / (n * n), r = c % (n * n), j = r / n, i = r % n;
        const double xi0 = -q + i * d, eta0 = -q + j * d;
        const double x1 = std::tan(xi0), x2 = std::tan(xi0 + d);
        const double y1 = std::tan(eta0), y2 = std::tan(eta0 + d);
        g.area[c] = R2 * (gnomonic_F(x2, y2) - gnomonic_F(x1, y2) - gnomonic_F(x2, y1) + gnomonic_F(x1, y1));
        const V3 c00 = sphere(p, xi0, eta0), c10 = sphere(p, xi0 + d, eta0);
        const V3 c11 = sphere(p, xi0 + d, eta0 + d), c01 = sphere(p, xi0, eta0 + d);
        g.edge_len[0 * ncol + c] = radius * arc(c10, c11);
        g.edge_len[1 * ncol + c] = radius * arc(c00, c01);
        g.edge_len[2 * ncol + c] = radius * arc(c01, c11);
        g.edge_len[3 * ncol + c] = radius * arc(c00, c10);
        const double xic = xi0 + 0.5 * d, etac = eta0 + 0.5 * d;
        centre[c] = sphere(p, xic, etac);
        g.sinlat[c] = centre[c].z;
        for (int s = 0; s < 4; ++s) {
            const V3 v = sphere(p, xic + 0.75 * d * di[s], etac + 0.75 * d * dj[s]);
            int pn;
            double a, b;
            locate(v, pn, a, b);
            int in = (int)std::floor((std::atan(a) + q) / d);
            int jn = (int)std::floor((std::atan(b) + q) / d);
            in = in < 0 ? 0 : (in >= n ? n - 1 : in);
            jn = jn < 0 ? 0 : (jn >= n ? n - 1 : jn);
            g.nbr[s * ncol + c] = pn * n * n + jn * n + in;
        }
    }
    // consistency: the neighbour across side s must see this column across exactly one side
    for (int c = 0; c < ncol; ++c) {
        for (int s = 0; s < 4; ++s) {
            const int cn = g.nbr[s * ncol + c];
            int found = -1, count = 0;
            for (int t = 0; t < 4; ++t)
                if (g.nbr[t * ncol + cn] == c) { found = t; ++count; }
            if (count != 1 || cn == c) {
                char buf[160];
                std::snprintf(buf, sizeof buf, "cubed-sphere connectivity broken at column %d side %d", c, s);
                return buf;
            }
            g.nbr_side[s * ncol + c] = found;
            g.cdist[s * ncol + c] = radius * arc(centre[c], centre[cn]);
        }
    }
    // horizontal faces: each listed once under its lower-numbered column, by (column, side)
    g.face_of.assign(4 * ncol, -1);
    g.faceL.clear();
    g.faceR.clear();
    g.faceSide.clear();
    for (int c = 0; c < ncol; ++c) {
        for (int s = 0; s < 4; ++s) {
            const int cn = g.nbr[s * ncol + c];
            if (c < cn) {
                const int f = (int)g.faceL.size();
                g.faceL.push_back(c);
                g.faceR.push_back(cn);
                g.faceSide.push_back(s);
                g.face_of[s * ncol + c] = f;
                g.face_of[g.nbr_side[s * ncol + c] * ncol + cn] = f;
            }
        }
    }
    if ((int)g.faceL.size() != 2 * ncol) return "cubed-sphere face count is not 2 ncol";
    return "";
}

std::string build_vgeom(const double* z, int nlev, VGeom& v) {
    v.nlev = nlev;
    v.dz.assign(nlev, 0.0);
    v.dzc.assign(nlev + 1, 0.0);
    for (int k = 0; k < nlev; ++k) {
        v.dz[k] = z[k + 1] - z[k];
        if (!(v.dz[k] > 0.0)) return "z_interfaces must be strictly increasing";
    }
    for (int kf = 1; kf < nlev; ++kf) v.dzc[kf] = 0.5 * (z[kf + 1] - z[kf - 1]);
    return "";
}

void level_coefficients(const HGeom& h, const VGeom& v, double cs_dt, LevelCoef& c) {
    const int ncol = h.ncol, nlev = v.nlev, nf = 2 * ncol;
    const double c2 = cs_dt * cs_dt;
    c.Th.assign((size_t)nlev * nf, 0.0);
    c.Tv.assign((size_t)(nlev + 1) * ncol, 0.0);
    for (int f = 0; f < nf; ++f) {
        const int L = h.faceL[f], R = h.faceR[f], s = h.faceSide[f];
        const double geo = h.edge_len[s * ncol + L] / h.cdist[s * ncol + L] * (c.muh.empty() ? 1.0 : c.muh[f]);
        for (int k = 0; k < nlev; ++k) {
            const double gf = 0.5 * (c.g[(size_t)k * ncol + L] + c.g[(size_t)k * ncol + R]);
            c.Th[(size_t)k * nf + f] = c2 * gf * geo;
        }
    }
    for (int kf = 1; kf < nlev; ++kf) {
        for (int col = 0; col < ncol; ++col) {
            const double gf = 0.5 * (c.g[(size_t)(kf - 1) * ncol + col] + c.g[(size_t)kf * ncol + col]);
            c.Tv[(size_t)kf * ncol + col] = c2 * gf * c.mu[(size_t)kf * ncol + col] / v.dzc[kf];
        }
    }
}

void restrict_mean(const HGeom& fine, const HGeom& coarse, int rows, const double* f, double* out) {
    const int ncf = fine.ncol, ncc = coarse.ncol;
    for (int k = 0; k < rows; ++k) {
        for (int C = 0; C < ncc; ++C) {
            double acc = 0.0;
            for (int q = 0; q < 4; ++q) {
                const int ch = child_col(fine.n, C, q);
                acc += fine.area[ch] * f[(size_t)k * ncf + ch];
            }
            out[(size_t)k * ncc + C] = acc / coarse.area[C];
        }
    }
}

void restrict_face_mean(const HGeom& fine, const HGeom& coarse, const double* f, double* out) {
    // children q = 2b + a of a coarse column lying on each side: E a = 1, W a = 0, N b = 1, S b = 0
    static const int on_side[4][2] = {{1, 3}, {0, 2}, {2, 3}, {0, 1}};
    const int ncf = fine.ncol, ncc = coarse.ncol;
    for (int F = 0; F < 2 * ncc; ++F) {
        const int C = coarse.faceL[F], s = coarse.faceSide[F];
        double acc = 0.0, wsum = 0.0;
        for (int t = 0; t < 2; ++t) {
            const int ch = child_col(fine.n, C, on_side[s][t]);
            const double w = fine.edge_len[s * ncf + ch];
            acc += w * f[fine.face_of[s * ncf + ch]];
            wsum += w;
        }
        out[F] = acc / wsum;
    }
}

}  // namespace mg
