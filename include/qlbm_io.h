/* Restart files (checkpoint and resume) of a single-domain solver.
 *
 * A file holds what ql_create needs and the state:
 *   line 1  "qlbm-checkpoint 1"
 *   line 2  one JSON object: Q, nx, length, dt, denseness, kn, bc ("periodic"
 *           or "fixed"), precision ("fp64" or "fp32"), pr_mode, pr_const,
 *           enskog, rho_ref, chi_mode, steps, time (= steps dt), ghost (18
 *           numbers: (rho, u, T) of cells -3, -2, -1, nx, nx+1, nx+2 for
 *           fixed ends, zeros for periodic ones), byte_order ("little")
 *   then    phi and theta, nx*Q doubles each, cell-major as ql_get_state
 *           gives them (an FP32 state is stored exactly, as doubles).
 * Numbers are written with 17 significant digits, so they read back to the
 * same doubles.  The scheme has no time-dependent forcing and the fixed ghost
 * cells come from the stored states, so a run resumed from a file continues
 * bitwise as the run that wrote it.  Host byte order must be little-endian
 * (x86-64 and AArch64 are).
 */
#ifndef QLBM_IO_H
#define QLBM_IO_H

#include "qlbm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Parameters of a restart file, as stored. */
typedef struct {
    int32_t Q;
    int32_t bc_kind;    /* QL_BC_PERIODIC or QL_BC_FIXED */
    int32_t precision;  /* QL_FP64 or QL_FP32 */
    int32_t pr_mode;
    int32_t enskog;
    int32_t chi_mode;
    int64_t nx;
    int64_t steps;
    double length, dt, denseness, kn, pr_const, rho_ref;
    double ghost[18];
} ql_checkpoint_info;

/* Steps the context has advanced: ql_step calls since ql_create, or since
 * the stored count for a context made by ql_load. */
ql_status ql_step_count(const ql_ctx *ctx, int64_t *steps);

/* Writes ctx's parameters, step count and state to path (through a
 * temporary file renamed into place, so a reader never sees a partial file).
 * Synchronises.  Errors: QL_EINVAL (null argument; the file cannot be
 * written, with the reason in ql_last_error), QL_ENOMEM, QL_ECUDA. */
ql_status ql_save(ql_ctx *ctx, const char *path);

/* Reads the parameters of a restart file without touching the GPU.  Errors:
 * QL_EINVAL (null argument, unreadable file, bad first line, a missing or
 * malformed field, a state size that does not match nx and Q),
 * QL_EUNSUPPORTED (big-endian host). */
ql_status ql_checkpoint_read_info(const char *path, ql_checkpoint_info *info);

/* Creates a context from a restart file: the stored parameters fix the
 * physics, precision and boundary; opts (may be NULL: device 0, the legacy
 * default stream, cudaMalloc) supplies device, stream and allocator, and
 * its precision, pr_mode, enskog, chi_mode, pr_const and rho_ref are
 * ignored.  The state and step count are the stored ones.  Errors: those of
 * ql_checkpoint_read_info and ql_create; *out is NULL on error. */
ql_status ql_load(const char *path, const ql_opts *opts, ql_ctx **out);

#ifdef __cplusplus
}
#endif

#endif /* QLBM_IO_H */
