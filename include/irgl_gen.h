/*
 * irgl_gen.h -- seeded synthetic CSR graph generator (input side only).
 *
 * This module produces the inputs that both the CUDA path (libirgl.so) and
 * the CPU oracle consume. It contains none of the traversal arithmetic: it
 * draws graphs, it never computes levels, distances or labels.
 *
 * Graph shapes follow the workload classes named for the worklist ForAll
 * (high-diameter meshes and R-MAT power-law graphs); the paper itself ships
 * no inputs (Sec. 1 names only the target GPUs).
 *
 * Randomness: every draw is counter-based, SplitMix64 (Vigna's published
 * mixing function) keyed by (seed, stream, index), so the output does not
 * depend on thread count, scheduling or host architecture.
 *
 * CSR layout written by every generator:
 *   row_ptr[0..n]   uint32, row_ptr[0] = 0, row_ptr[n] = m, non-decreasing
 *   col[0..m)       uint32 destination ids, strictly increasing within a row
 *                   (no duplicates, no self-loops)
 *   w[0..m)         int32 weights in [1, 100] when the caller passes w != NULL
 * The caller owns all buffers; `cap` is the capacity of col/w in elements.
 * Return value: m (>= 0) on success, or a negative code:
 *   -1 invalid argument, -2 capacity too small, -3 out of host memory.
 */
#ifndef IRGL_GEN_H
#define IRGL_GEN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* One counter-based draw: SplitMix64 mixing of (seed, stream, index). */
uint64_t irglgen_draw(uint64_t seed, uint64_t stream, uint64_t index);

/* rows x cols 4-neighbour mesh, vertex id = r*cols + c.
 * del_frac:   exactly round(del_frac * E) of the E undirected grid edges are
 *             deleted (both directions), chosen by seeded keys.
 * extra_frac: round(extra_frac * rows*cols) distinct seeded vertices each get
 *             one extra undirected edge to an offset (dr,dc) != 0 with
 *             |dr|+|dc| <= radius inside the mesh, redrawn on a duplicate.
 * With del_frac = extra_frac = 0 this is the plain grid.
 * Weights (if w != NULL): one draw per undirected edge, same both ways. */
int64_t irglgen_mesh(uint32_t rows, uint32_t cols, uint64_t seed,
                     double del_frac, double extra_frac, uint32_t radius,
                     uint32_t* row_ptr, uint32_t* col, int32_t* w,
                     uint64_t cap);

/* R-MAT: ef * 2^scale edge samples, each bit level picks a quadrant with
 * probabilities (a, b, c, 1-a-b-c); vertex ids then go through a seeded
 * permutation; self-loops dropped, duplicates merged, rows sorted.
 * Weights (if w != NULL): a draw per directed (u, v) pair, uniform [1,100].
 * nthreads <= 0 uses the hardware concurrency. */
int64_t irglgen_rmat(uint32_t scale, uint32_t ef, double a, double b, double c,
                     uint64_t seed, int nthreads,
                     uint32_t* row_ptr, uint32_t* col, int32_t* w,
                     uint64_t cap);

#ifdef __cplusplus
}
#endif
#endif /* IRGL_GEN_H */
