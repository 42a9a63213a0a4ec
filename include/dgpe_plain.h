/*
 * dgpe_plain.h -- comparison step (libdgpe_plain.so): the same real-time
 * split step as dgpe_step, built the way the paper's programs build it
 * (arXiv:1601.04640, "Summary of revisions": separate grid-stride kernels,
 * cuFFT real-to-complex / complex-to-real transforms for the dipolar term,
 * Crank-Nicolson recursions with one thread per grid line, forward-sweep
 * values in a temporary array).  It exists to be timed beside the fused path;
 * nothing in libdgpe.so calls it.
 *
 * Parameters and psi layout as in dgpe.h (mode must be DGPE_REAL; precision
 * DGPE_FP64 uses cufftExecD2Z/Z2D, DGPE_FP32_BULK cufftExecR2C/C2R and FP32
 * arithmetic throughout).  psi buffers are host FP64 interleaved complex of
 * nx*ny(*nz) values.  Every call returns DGPE_OK or a negative DGPE_E* code;
 * dgpe_plain_last_error() gives the text.  The library owns its device
 * buffers and cuFFT plans; the caller owns the stream.
 */
#ifndef DGPE_PLAIN_H
#define DGPE_PLAIN_H

#include "dgpe.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dgpe_plain_solver *dgpe_plain_t;

int dgpe_plain_create(const dgpe_params *p, void *cuda_stream, dgpe_plain_t *out);
void dgpe_plain_destroy(dgpe_plain_t h);
int dgpe_plain_set_psi(dgpe_plain_t h, const double *psi);   /* synchronous */
int dgpe_plain_get_psi(dgpe_plain_t h, double *psi);         /* synchronises */
int dgpe_plain_step(dgpe_plain_t h, int n);                  /* asynchronous */
const char *dgpe_plain_last_error(void);

#ifdef __cplusplus
}
#endif

#endif
