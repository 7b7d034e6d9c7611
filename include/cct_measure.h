/* cct_measure.h -- measurement aid of libcct (no counterpart in the paper).
 *
 * The walk of Sec. 5.1 reads one 32-byte triangle record per step at a
 * data-dependent address.  Its roofline denominator is therefore the rate at
 * which the GPU serves random 32-byte sectors from a table of the walked
 * table's size -- from L2 when the table fits there (129 MB on GB300), from
 * HBM otherwise.  This call measures that rate with independent (not
 * pointer-chased) random loads, so it is the ceiling the dependent walk can
 * approach but not exceed.
 */
#ifndef CCT_MEASURE_H
#define CCT_MEASURE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Allocates a device table of table_bytes (rounded down to 32-byte records,
 * at least one), fills it, then times `reps` launches of a kernel in which
 * every thread of a full-occupancy grid issues independent 256-bit loads at
 * hashed record indices, `loads` loads in total per launch.  Writes the mean
 * launch time (ms, CUDA events on `stream`) and the achieved bytes per second
 * (32 bytes per load) to *ms_per_launch and *bytes_per_s.  Frees the table
 * before returning (synchronises `stream`).
 * Errors: CCT_ERR_INVALID_ARGUMENT (bad size or null output),
 * CCT_ERR_OUT_OF_MEMORY, CCT_ERR_CUDA. */
int cct_measure_gather(size_t table_bytes, int64_t loads, int32_t reps, void* stream, float* ms_per_launch,
                       double* bytes_per_s);

#ifdef __cplusplus
}
#endif

#endif /* CCT_MEASURE_H */
