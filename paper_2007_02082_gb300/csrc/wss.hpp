// Wall shear stress at the Lagrangian points (Sec. 2.6) by second-order DC-PSE
// derivatives; see wss.cu.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "ibmove.hpp"

namespace ibg {

// cutoff radius of the DC-PSE point cloud, in units of the largest finest spacing
constexpr double WSS_RADIUS = 3.5;

// wss[p] (and grad[p][i][j] = d u_i / d x_j when grad is not null) at points
// 0..M-1 from the slot-layout velocity u ([3][ns]); mu = nu_rho.  *err is set
// to 1 when a point has too few fluid nodes for the nine moment conditions.
void wss_compute(const MoveGrid& G, const double hf[3], int64_t M, const double* X, const double* UB,
                 const double* nrm, const double* u, int64_t ns, double nu_rho, double* wss, double* grad,
                 int32_t* err, cudaStream_t st);

}  // namespace ibg
