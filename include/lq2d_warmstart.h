/* Learned warm start for the PCG solver of lq2d.h.
 *
 * Algorithm 1 (PCGM) accepts any initial iterate delta^(0) and sets
 * r^(0) = r_delta - Delta delta^(0); the paper starts from zero.  This part
 * adds a small convolutional network over the K x N grid of subsystems that
 * proposes delta^(0) from the instance's initial states x0 and its coupling
 * scale c; the solver then runs from that iterate (lq2d_solve_device,
 * argument d_delta0) and, as from a zero start, stops only on the tolerance,
 * so a poor guess costs iterations, never accuracy.
 *
 * Network: `layers` 3x3 convolutions with zero padding, ReLU between layers,
 * none after the last; input channels x0_{i,j} (n) and c (1); `channels`
 * channels in every hidden layer; output (T+1) n channels per node, mapped
 * to the costate guess by
 *     delta0[t][i*N + j][k] = sigma * yhat[t*n + k][i][j].
 * Weights are kept in FP32 (the Adam master copy) and used in the forward
 * and backward passes as bfloat16 (round to nearest even); activations and
 * accumulation are FP32.  Training minimises the mean squared error between
 * yhat and delta* / sigma, delta* the solver's costates, with Adam (Kingma
 * and Ba 2015, Algorithm 1; beta1 0.9, beta2 0.999, eps 1e-8).
 *
 * Parameter vector (FP32, host copies in this layout): for each layer l in
 * order, its weights [C_out][C_in][3][3] row-major, then its bias [C_out].
 *
 * Device buffers are caller-owned, FP64, in the layouts of lq2d.h:
 * x0 [batch][K*N][n], delta [batch][T+1][K*N][n].  Every call returns after
 * its work on `stream` is complete.  Errors: LQ2D_EINVAL (bad argument,
 * batch above max_batch), LQ2D_ENOMEM, LQ2D_ECUDA; text via
 * lq2d_last_error(). */
#ifndef LQ2D_WARMSTART_H
#define LQ2D_WARMSTART_H

#include "lq2d.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lq2d_wsnet lq2d_wsnet;

/* Allocates a network for K x N grids over horizon T with state dimension n
 * (1..8), `layers` >= 1 convolutions of `channels` (1..256) hidden channels,
 * batches of up to max_batch instances and output scale sigma > 0.  The
 * parameters are zero until lq2d_wsnet_set_params. */
int lq2d_wsnet_create(lq2d_wsnet **out, int K, int N, int T, int n, int channels, int layers,
                      int max_batch, double sigma);

/* Number of FP32 parameters (length of the vector described above). */
int lq2d_wsnet_param_count(const lq2d_wsnet *net, long long *count);

/* Copies the FP32 parameters from / to host memory.  set_params also clears
 * the Adam moments and step count. */
int lq2d_wsnet_set_params(lq2d_wsnet *net, const float *params);
int lq2d_wsnet_get_params(const lq2d_wsnet *net, float *params);

/* delta0 for `batch` instances: d_x0 [batch][K*N][n], coupling [batch] (host
 * array), d_delta0 [batch][T+1][K*N][n] (written). */
int lq2d_wsnet_forward_device(lq2d_wsnet *net, int batch, const double *d_x0, const double *coupling,
                              double *d_delta0, void *stream);

/* Loss of the network on `batch` instances with targets d_target
 * [batch][T+1][K*N][n] (the solver's costates), and, when grads is not NULL,
 * its gradient with respect to the parameters (host array, parameter-vector
 * layout).  The parameters are not changed. */
int lq2d_wsnet_loss_grad_device(lq2d_wsnet *net, int batch, const double *d_x0, const double *coupling,
                                const double *d_target, double *loss, float *grads, void *stream);

/* One training step: the loss and gradient as above, then one Adam update
 * of the parameters with learning rate lr.  *loss (may be NULL) is the loss
 * before the update. */
int lq2d_wsnet_train_step_device(lq2d_wsnet *net, int batch, const double *d_x0, const double *coupling,
                                 const double *d_target, double lr, double *loss, void *stream);

void lq2d_wsnet_destroy(lq2d_wsnet *net);

#ifdef __cplusplus
}
#endif

#endif /* LQ2D_WARMSTART_H */
