/* Measurement utilities of liblmspdhg.so used only by the benchmark
 * (bench.py): they have no counterpart in the paper and are not part of the
 * LM-SPDHG interface of lmspdhg.h.  They give the benchmark's in-run L2
 * peaks for gather and atomic traffic and the exact traversal counts behind
 * its algorithmic byte counts.  Conventions as in lmspdhg.h (LM_* status,
 * lm_last_error, device pointers owned by the caller). */
#ifndef LM_MEASURE_H
#define LM_MEASURE_H

#include "lmspdhg.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Exact traversal counts of an event list: samples with a non-zero TOF
 * weight and an in-grid neighbour, and in-grid neighbour touches (each touch
 * is one 4-byte image read in a forward projection and one 4-byte atomic add
 * in a back-projection).  ws: device, >= 16 bytes.  Synchronous. */
int lm_traversal_stats(const lm_scanner* sc, const lm_grid* grid, const lm_tof* tof, const lm_events* ev,
                       void* ws, size_t ws_bytes, int64_t* n_samples, int64_t* n_touches, void* stream);

/* L2 throughput probe on the caller's device buffer (use one that fits in
 * L2): mode 0 coalesced 16-byte reads, 1 coalesced float atomic adds, 2
 * random 4-byte reads, 3 random float atomic adds; *gbs_out = payload GB/s
 * over `iters` passes.  The buffer is overwritten.  Modes 4 and 5 probe
 * shared memory instead (random 4-byte reads / float atomic adds on a 32 KB
 * array per block, 64 x iters accesses per thread; buf only receives a
 * guard value).  Synchronous. */
int lm_probe_l2(void* buf, size_t bytes, int32_t mode, int32_t iters, double* gbs_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LM_MEASURE_H */
