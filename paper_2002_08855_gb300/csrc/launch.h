// Host-side launchers of the IB-LBM kernels (internal to libibmlbm.so).
#pragma once

#include <string>

#include "common.cuh"

namespace ibmlbm {

// fault words of the bounds-checked build, per translation unit (0 in the ordinary build)
unsigned long long check_fault_lbm();
unsigned long long check_fault_ibm();
unsigned long long check_fault_pairs();

cudaError_t launch_lbm_step(const LbmArgs& A, int D, int parity, cudaStream_t s);
int lbm_step_launches(const Geo& g, int D, int parity, int store);  // kernels launch_lbm_step launches
bool lbm_step_vector(const Geo& g, int D, int store);  // launch_lbm_step uses the vector kernel
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
size_t spread_smem(int D, int nl, int box);  // of the kernel launch_ibm_spread uses
cudaError_t prepare_ibm_spread(int D, size_t smem);  // once, before any capture
cudaError_t launch_ibm_forces(const IbmArgs& A, cudaStream_t s);
cudaError_t launch_regen(const RegenArgs& A, int init, cudaStream_t s);

// pair search: cell buckets, neighbour lists, contact forces (and the particle update)
cudaError_t launch_pair_cells(const PairArgs& A, cudaStream_t s);   // memset + 1 kernel
cudaError_t launch_pair_contacts(const PairArgs& A, cudaStream_t s);
cudaError_t launch_pair_search_lists(const PairArgs& A, cudaStream_t s);  // partner lists only
cudaError_t launch_pair_forces(const PairArgs& A, cudaStream_t s);        // forces (and update)
cudaError_t launch_pair_compact(const PairArgs& A, int* pairs, long long cap, cudaStream_t s);
cudaError_t launch_scan(const int* in, int* out, int n, cudaStream_t s);

// fused launches over the members of a 2D batch (block counts per member, then the
// launches; see Fuse in common.cuh)
unsigned lbm_step_blocks(const Geo& g, int store);
unsigned lbm_edge_blocks(const Geo& g, int D);
cudaError_t launch_lbm_nee(const LbmArgs& A, int D, int parity, cudaStream_t s);
int tile_shape_count();
void tile_shape(int s, int store, int* k, int* w, int* persist);
int tile_count(const Geo& g, int s);
cudaError_t launch_lbm_step_tiles(int shape, const LbmArgs* args, const int* first, int n, int total,
                                  const Fuse& FE, unsigned eblocks, int store, int parity, cudaStream_t s);
cudaError_t launch_lbm_step_fused(const Fuse& F, unsigned blocks, const Fuse& FE, unsigned eblocks,
                                  int store, int parity, cudaStream_t s);
size_t ibm_box2_smem(int box);
unsigned ibm_warp_blocks(int np);
unsigned ibm_lane_blocks(int np);
unsigned ibm_half_blocks(int np);  // interior sums: a half-warp per particle
cudaError_t launch_ibm_interp_fused(const Fuse& F, unsigned blocks, size_t smem, int m, int parity,
                                    int store, cudaStream_t s);
cudaError_t launch_ibm_spread_fused(const Fuse& F, unsigned blocks, size_t smem, cudaStream_t s);
cudaError_t launch_ibm_forces_fused(const Fuse& F, unsigned blocks, cudaStream_t s);
cudaError_t launch_regen_fused(const Fuse& F, unsigned blocks, cudaStream_t s);
unsigned pair_clear_blocks(const PairArgs& A);
unsigned pair_thread_blocks(int n, int b);
unsigned pair_warp_blocks(int n);
cudaError_t launch_pairs_fused(const Fuse& Fc, unsigned bc, const Fuse& Fi, unsigned bi,
                               const Fuse& Fs, unsigned bs, const Fuse& Ff, unsigned bf,
                               cudaStream_t s);
// persistent (cooperative) kernels of a batched step, phases separated by bounded grid
// barriers: the IBM phases (regeneration, MDF iterations, forces) and the contact
// phases (clear, insert, search, force and update).  prepare: only raise the kernel's
// shared-memory limit (once, before any stream capture).
cudaError_t launch_ibm_batch(const IbmBatch& P, int parity, int store, size_t smem, cudaStream_t s,
                             bool prepare);
cudaError_t launch_pairs_batch(const PairBatch& P, cudaStream_t s);

// sets the calling thread's text for ibm_lbm_last_error()
void set_last_error(const std::string& msg);

}  // namespace ibmlbm
