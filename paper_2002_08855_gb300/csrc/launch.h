// Host-side launchers of the IB-LBM kernels (internal to libibmlbm.so).
#pragma once

#include <string>

#include "common.cuh"

namespace ibmlbm {

cudaError_t launch_lbm_step(const LbmArgs& A, int D, int parity, cudaStream_t s);
cudaError_t launch_lbm_moments(const LbmArgs& A, int D, int parity, cudaStream_t s);
cudaError_t launch_lbm_fields(const LbmArgs& A, int D, int parity, double* p, double* u,
                              cudaStream_t s);
cudaError_t launch_lbm_get(const LbmArgs& A, int D, int parity, float* out, cudaStream_t s);
cudaError_t launch_lbm_put(const LbmArgs& A, int D, int parity, const float* in,
                           cudaStream_t s);
cudaError_t launch_lbm_equilibrium(const LbmArgs& A, int D, int parity, const double* p,
                                   const double* u, cudaStream_t s);

cudaError_t launch_ibm_interp(const IbmArgs& A, int m, cudaStream_t s);
cudaError_t launch_ibm_spread(const IbmArgs& A, cudaStream_t s);
size_t ibm_spread_smem(int D, int nl, int box);
cudaError_t prepare_ibm_spread(int D, size_t smem);  // once, before any capture
cudaError_t launch_interior_momentum(const IbmArgs& A, cudaStream_t s);
cudaError_t launch_particle_update(const PartArgs& A, int mode, int have_prev, cudaStream_t s);

// pair search: cell lists by counting sort, neighbour lists and contact forces
cudaError_t launch_pair_cells(const PairArgs& A, cudaStream_t s);   // 3 kernels
cudaError_t launch_pair_contacts(const PairArgs& A, cudaStream_t s);
cudaError_t launch_pair_compact(const PairArgs& A, int* pairs, long long cap, cudaStream_t s);
cudaError_t launch_scan(const int* in, int* out, int n, cudaStream_t s);

// sets the calling thread's text for ibm_lbm_last_error()
void set_last_error(const std::string& msg);

}  // namespace ibmlbm
