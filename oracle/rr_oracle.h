/*
 * rr_oracle.h -- sequential CPU oracle for the improved red-rec planner and
 * the batching routine of Afiouni et al., "Efficient algorithms to solve atom
 * reconfiguration problems III" (arXiv 2504.06182), Alg. 1, 2 and 4.
 *
 * TEST INFRASTRUCTURE ONLY. The oracle is the slow, plain statement of what
 * the planner computes; the tests, the smoke check and the benchmark's CPU
 * baseline leg are its only users. It shares no code, header, table or
 * constant with the CUDA library, and the library never calls it.
 *
 * Conventions (own copy, deliberately not shared with the library header):
 *   grid    m*n bytes, row-major, 1 = occupied trap.
 *   rect    half-open target rectangle rows [r0, r1), columns [c0, c1).
 *   move    4 int32 (src_row, src_col, dst_row, dst_col); an L-shaped path
 *           that first runs along row src_row to column dst_col, then along
 *           column dst_col to dst_row.
 *   op      3 int32 (dir, first, count); dir 0 = row-1, 1 = row+1,
 *           2 = col-1, 3 = col+1; members[first .. first+count) are the ids
 *           of the moves that advance one elementary step in this batch.
 * Return codes: 0 ok, 1 infeasible (no moves), -1 bad argument,
 *   -2 capacity (required sizes written), -5 out of memory, -6 internal
 *   invariant broken (a bug in the oracle).
 */
#ifndef RR_ORACLE_H
#define RR_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Optimal contiguous window (Sec. III.A, exact 1D with contiguous targets):
 * sources s[0..K) sorted ascending (repeats allowed: several tokens on one
 * vertex, Sec. III.A "Generalized assignment"), targets r0 .. r0+h-1, K >= h.
 * Returns the window start w minimising sum_k |s[w+k] - (r0+k)|, smallest w on
 * ties; -1 on bad arguments. */
int rro_window(const int32_t *s, int K, int r0, int h);

/* Receiver split (Sec. III.C, redistribution as a 1D instance): mandatory
 * source rows mand[0..nm), optional pool rows split into top[0..nt) (rows <
 * r0, any order) and bot[0..nb) (rows >= r1, any order); choose x pool atoms
 * so that the mandatory plus chosen rows, sorted and matched to r0..r0+h-1
 * (nm + x = h), have minimum total distance. Only "a nearest-from-top plus
 * x-a nearest-from-bottom" choices are considered; largest a on ties.
 * Returns a, or -1 on bad arguments. *cost_out (may be NULL) gets the cost. */
int rro_split(const int32_t *mand, int nm, const int32_t *top, int nt,
              const int32_t *bot, int nb, int x, int r0, int h,
              int64_t *cost_out);

/* The planner (Alg. 1 in its parallel-variant ordering, Sec. III.D).
 * moves: cap*4 int32. sigma_out: n int32 surpluses after the column solves
 * (may be NULL). events: cap_ev*5 int32 (case, donor, receiver, x, a) per
 * pairing iteration (may be NULL). */
int rro_plan(const uint8_t *grid, int m, int n, int r0, int c0, int r1, int c1,
             int32_t *moves, int64_t cap, int64_t *n_moves,
             int32_t *sigma_out, int32_t *events, int64_t cap_ev,
             int64_t *n_events);

/* rro_plan with a geometry mode: strict = 0 solves columns outside the
 * target columns with their own reservoir cells as virtual targets (their
 * band-row atoms become donatable); strict = 1 leaves them as they are, so
 * only their reservoir-row atoms are donatable (the paper's donors donate
 * reservoir atoms only, Sec. III.C). With a full-width target both are the
 * paper's algorithm. */
int rro_plan_mode(const uint8_t *grid, int m, int n, int r0, int c0, int r1, int c1,
                  int32_t *moves, int64_t cap, int64_t *n_moves,
                  int32_t *sigma_out, int32_t *events, int64_t cap_ev,
                  int64_t *n_events, int strict);

/* The bird planner (Alg. 2, Sec. III.E): red-rec's column phase, then the
 * unsolved columns left to right, each filled through its generalised 1D
 * instance over every token of the grid. moves: cap*4 int32. units:
 * cap_units*3 int32 (receiver column, tokens taken from above the band,
 * tokens taken from below it) per receiver (may be NULL). */
int rro_bird(const uint8_t *grid, int m, int n, int r0, int c0, int r1, int c1,
             int32_t *moves, int64_t cap, int64_t *n_moves,
             int32_t *units, int64_t cap_units, int64_t *n_units);

/* rro_bird with the geometry mode of rro_plan_mode. */
int rro_bird_mode(const uint8_t *grid, int m, int n, int r0, int c0, int r1, int c1,
                  int32_t *moves, int64_t cap, int64_t *n_moves,
                  int32_t *units, int64_t cap_units, int64_t *n_units, int strict);

/* The same planner stopped after its first max_units receiver units (the
 * column phase and a leading sample of the move list, for grids too large
 * to plan completely this way). */
int rro_bird_prefix(const uint8_t *grid, int m, int n, int r0, int c0, int r1, int c1,
                    int32_t *moves, int64_t cap, int64_t *n_moves, int64_t max_units);

/* The batching routine (Alg. 4 with the local constraint set of Sec. IV).
 * ops: cap_ops*3 int32; members: cap_members int32. */
int rro_batch(const int32_t *moves, int64_t n_moves, int m, int n,
              int32_t *ops, int64_t cap_ops, int32_t *members,
              int64_t cap_members, int64_t *n_ops, int64_t *n_members);

/* Same routine, stopped after the first max_ops batches (a leading sample of
 * the batch list for inputs too large to batch completely). */
int rro_batch_prefix(const int32_t *moves, int64_t n_moves, int m, int n,
                     int64_t max_ops, int32_t *ops, int64_t cap_ops,
                     int32_t *members, int64_t cap_members, int64_t *n_ops,
                     int64_t *n_members);

#ifdef __cplusplus
}
#endif
#endif
