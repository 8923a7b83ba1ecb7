// geom.h -- host-side geometry of the immersed body: velocity grid and dual
// boxes, cell classes, links (ghost cell, donor cell, auxiliary cell, intersect
// point, normal, shifted point), surface-cell lists and the incident-side
// measure of the velocity boxes cut by the wall plane.
//
// Definitions follow arXiv 2512.20252 Sec. 3.2.1 (cell and point classes),
// Eqs. sp/fsp/fw/extrapolation 2 (the coefficients along the link axis) and
// Sec. 3.2.3 (velocity-space cut cells).  All FP64, built once per body.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/ibdvm.h"

namespace ibdvm {

struct Link {
  int ghost;      // ghost cell
  int gidx;       // index of the ghost in the ghost list
  int donor;      // fluid face neighbour of the ghost
  int aux;        // auxiliary cell beyond the donor, -1 when it is not a fluid cell
  int axis, side; // side = sign of (x_donor - x_ghost) along axis
  double xw[3];   // intersect point
  double nw[3];   // unit normal into the gas
  // linear interpolation coefficients along the link axis (y = coordinate on the axis)
  double c_sp;    // (y_sp - y_d) / (y_ac - y_d), 0 without an auxiliary cell   (Eq. fsp)
  double c_iw;    // (y_w - y_sp) / (y_g - y_sp)                                  (Eq. fw)
  double c_gc;    // (y_g - y_sp) / (y_w - y_sp)                                  (Eq. extrapolation 2)
};

struct Geom {
  // physical grid
  int dim = 2, ncomp = 2;
  int n[3] = {1, 1, 1};
  double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1}, dx[3] = {1, 1, 1};
  long long ncell = 0;
  // velocity grid
  int rule = 0;
  int nvx[3] = {1, 1, 1};
  int nv = 0, nvp = 0;          // nodes, nodes padded to a multiple of kVelPad
  std::vector<double> xi;       // [nv][3]
  std::vector<double> w;        // [nv]
  std::vector<double> blo, bhi; // [nv][3] dual boxes
  // gas
  double mu0 = 0, dt = 0, Uinf[3] = {0, 0, 0};
  ibdvm_gas_desc gas{};
  // body
  ibdvm_body_desc body{};
  std::vector<double> verts;
  // classification and links
  std::vector<uint8_t> type;      // [ncell]
  std::vector<int> ghosts;        // ghost cells, ascending
  std::vector<int> ghost_first;   // first link of each ghost
  std::vector<int> ghost_nlinks;
  std::vector<Link> links;
  std::vector<int> surf_off;      // [nghost+1]
  std::vector<int> surf_cell;     // [nsurf]
  std::vector<double> wg;         // [nlink][nv] incident-side measure
  long long nfluid = 0;
};

constexpr int kVelPad = 64;

// Builds the velocity grid and gas constants; no body (all cells fluid).
bool build_grid(const ibdvm_grid_desc &g, const ibdvm_vgrid_desc &v, const ibdvm_gas_desc &gas,
                Geom &out, std::string &err);
// Places a body into a grid built by build_grid.
bool place_body(const ibdvm_body_desc &b, Geom &G, std::string &err);

// Closed-form measures of a velocity box on the incident side {xi.n <= 0}.
double incident_area_2d(const double *lo, const double *hi, const double *n);
double incident_volume_3d(const double *lo, const double *hi, const double *n);

// Cell centre coordinate along axis a (exactly mirror-symmetric about the
// domain centre).
double cell_coord(const Geom &G, int a, int i);

} // namespace ibdvm
