// Host-side cubed-sphere hierarchy and operator coefficients (FP64), built once by
// mg_setup before anything is uploaded to the GPU.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace mg {

// Horizontal geometry and connectivity of one cubed-sphere level C_n.
struct HGeom {
    int n = 0;
    int ncol = 0;
    std::vector<double> area;        // [ncol] cell area on the sphere of radius R
    std::vector<double> sinlat;      // [ncol] sine of the latitude of the cell centre (axis z)
    std::vector<int32_t> nbr;        // [4][ncol] neighbour column across side E, W, N, S
    std::vector<int32_t> nbr_side;   // [4][ncol] side of the neighbour that faces this column
    std::vector<double> edge_len;    // [4][ncol] length of the shared edge
    std::vector<double> cdist;       // [4][ncol] great-circle distance between centres
    std::vector<int32_t> face_of;    // [4][ncol] horizontal face index of each side
    std::vector<int32_t> faceL;      // [2 ncol] owning (lower-numbered) column of each face
    std::vector<int32_t> faceR;      // [2 ncol] the other column
    std::vector<int32_t> faceSide;   // [2 ncol] side of faceL the face lies on
};

// Builds C_n; returns an empty string or an error message.
std::string build_hgeom(int n, double radius, HGeom& out);

// Vertical grid shared by every level.
struct VGeom {
    int nlev = 0;
    std::vector<double> dz;    // [nlev] layer depths
    std::vector<double> dzc;   // [nlev+1] centre-to-centre distance at face kf (0 at kf=0,nlev)
};

std::string build_vgeom(const double* z_if, int nlev, VGeom& out);

// Coefficients of the Helmholtz operator on one level, in face form:
//   a_h(k, c, side) = Th[k][face_of[side][c]] / area[c]   (Th includes muh of the face)
//   a_up(k, c)      = Tv[k+1][c] / dz[k],   a_dn(k, c) = Tv[k][c] / dz[k]
struct LevelCoef {
    std::vector<double> Th;    // [nlev][2 ncol] (c_s dt)^2 g_f muh_f l_f / d_f
    std::vector<double> Tv;    // [nlev+1][ncol] (c_s dt)^2 g_f mu_f / dzc_f, 0 at kf = 0, nlev
    std::vector<double> g;     // [nlev][ncol] background factors on this level
    std::vector<double> mu;    // [nlev+1][ncol] vertical-face mass factors on this level
    std::vector<double> muh;   // [2 ncol] horizontal-face mass factors (empty: all 1)
};

void level_coefficients(const HGeom& h, const VGeom& v, double cs_dt, LevelCoef& c);

// Volume-weighted mean of the 4 children of every coarse column, level by level:
// out[k][C] = sum_ch area_ch f[k][ch] / area_C (same layer depth on both levels).
void restrict_mean(const HGeom& fine, const HGeom& coarse, int rows, const double* f,
                   double* out);

// Edge-length-weighted mean of the two fine faces that make up every coarse horizontal
// face: f [2 ncol_fine] -> out [2 ncol_coarse] (level-independent face fields).
void restrict_face_mean(const HGeom& fine, const HGeom& coarse, const double* f, double* out);

// Children of coarse column C = (p, J, I): q = 2b + a -> fine (p, 2J + b, 2I + a).
inline int32_t child_col(int n_fine, int C, int q) {
    const int nc = n_fine / 2;
    const int p = C / (nc * nc), r = C % (nc * nc), J = r / nc, I = r % nc;
    return p * n_fine * n_fine + (2 * J + (q >> 1)) * n_fine + 2 * I + (q & 1);
}

}  // namespace mg
