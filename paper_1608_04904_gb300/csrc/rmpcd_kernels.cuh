// rmpcd_kernels.cuh -- host-side launchers of the sm_103a kernels (internal).
#pragma once

#include <vector>

#include "rmpcd_common.cuh"

namespace rmpcd {

// Options of one cell pass (bit mask).
enum CellPassOpt {
    CP_FLIGHT = 1,    // records not marked PROP fly over tau when gathered
    CP_COLLIDE = 2,   // SRD / MPC-AT / virtual-particle collision
    CP_REACT = 4,     // bulk B -> A reaction
    CP_NEXT = 8,      // classify and bin every written record for the next collision
    CP_OBS = 16,      // per-tile observable partial sums
    CP_WRITE = 32,    // write the gathered (sorted) records to the output buffer
    CP_ADVANCE = 64   // advance the device step after the pass (fused intervals)
};

struct CellPassArgs {
    int opts;
    uint32_t step;     // collision index: grid shift, rotation axes, reactions (STEP_DEVICE: Ctl::step)
    int cur;           // count / bucket buffer consumed
    int nxt;           // count / bucket buffer filled by CP_NEXT
    int rin, rout;     // record buffers
};

enum ParticleMode { PM_STREAM = 0, PM_BIN = 1, PM_PRIME = 2 };

void launch_cellpass(bool mixed, const Dev &d, const CellPassArgs &a, cudaStream_t s);
// Set the device step (Ctl::step) on the stream.
void launch_set_step(const Dev &d, uint32_t step, cudaStream_t s);
// atomicMax of the largest count of count buffer b into d.maxcnt.
void launch_count_max(const Dev &d, int b, cudaStream_t s);
void launch_particles(bool mixed, const Dev &d, int mode, uint32_t step, int rbuf, int bbuf, cudaStream_t s);
// cs: CTAs per replica cluster, one of MD_CLUSTER_SIZES (results do not depend on it)
extern const int MD_CLUSTER_SIZES[4];
void launch_md(bool mixed, const Dev &d, uint32_t step, int rbuf, int bbuf, int do_bin, int cs, cudaStream_t s);
// Sub-steps [s0, s1) of the general MD kernel's interval (s1 < 0: to its end;
// see rmpcd_md_substep); the colloid state between calls lives in
// d.md_col_save (md_col_state_bytes per replica).
void launch_md_range(bool mixed, const Dev &d, uint32_t step, int rbuf, int bbuf, int do_bin, int cs, int s0, int s1,
                     cudaStream_t s);
size_t md_col_state_bytes(bool mixed);
// Few-colloid variant (every replica: at most MD_FAST_NC colloids, no
// colloid-colloid potential); bit-identical results to launch_md.
constexpr int MD_FAST_NC = 2;
// cs: 1, 2, 4, 8 or 16 (16 when md_fast_max_cluster allows it)
void launch_md_fast(bool mixed, const Dev &d, uint32_t step, int rbuf, int bbuf, int do_bin, int cs, cudaStream_t s);
int md_fast_max_cluster(bool mixed);
// The wide MD kernel (mixed path, many colloids): one cooperative launch of
// `grid` CTAs per listed replica; md_wide_grid() gives the co-resident grid.
void launch_md_wide(const Dev &d, const std::vector<int> &reps, int grid, uint32_t step, int rbuf, int bbuf,
                    int do_bin, cudaStream_t s);
int md_wide_grid();
// Rigid bead bodies: one CTA per replica (replicas without a body return at
// once); nb_max = the most beads of any body.  prepare_md_body sets the
// kernel's shared-memory limit for nb_max (not a stream operation).
// grid_bytes: shared-memory room for the lookup grids (md_body_grid_room;
// 0: read from global memory).
void launch_md_body(bool mixed, const Dev &d, int nb_max, int grid_bytes, uint32_t step, int rbuf, int bbuf,
                    int do_bin, cudaStream_t s);
cudaError_t prepare_md_body(bool mixed, int nb_max, int grid_bytes);
int md_body_grid_room(bool mixed, int nb_max, long long grid_entries_max);
// Bead networks (FP64 path): one CTA per replica (replicas without a network
// return at once) with `smem` bytes of dynamic shared memory
// (md_network_smem of the largest network; prepare_md_network sets the
// kernel's limit, not a stream operation).
size_t md_network_smem(int nb, int nl, int ncol);
cudaError_t prepare_md_network(size_t smem);
void launch_md_network(const Dev &d, size_t smem, uint32_t step, int rbuf, int bbuf, int do_bin, cudaStream_t s);
void launch_set_state(bool mixed, const Dev &d, int replica, int n, const double *x, const double *v,
                      const uint8_t *flags, int rbuf, cudaStream_t s);
void launch_get_state(bool mixed, const Dev &d, int replica, int n, int rbuf, double *x, double *v, uint8_t *flags,
                      uint32_t *id, int32_t *cell, int has_sort, uint32_t sort_step, cudaStream_t s);
void launch_obs_reduce(const Dev &d, cudaStream_t s);
// Gather a fused run's records (rows and overflow of buffer b, near area) into
// the flat slots of buffer fbuf, unsorted; fill[n_rep] zeroed by the caller
// counts them (4 launches).
void launch_flatten(bool mixed, const Dev &d, int b, int fbuf, int *fill, cudaStream_t s);
// Slab profile of one replica (n particles) into acc[n_bins * PROF_FIELDS] (zeroed by the caller).
void launch_profile(bool mixed, const Dev &d, int replica, int n, int rbuf, int axis, int n_bins,
                    unsigned long long *acc, cudaStream_t s);
size_t cellpass_smem(bool mixed);

}  // namespace rmpcd
