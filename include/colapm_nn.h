/*
 * colapm_nn.h -- learned displacement correction in libcolapm.so.
 *
 * The paper has no learned component. This network stands in for a fine-mesh, many-step COLA
 * run: it maps the final displacement field Psi of a coarse, few-step run (3 channels on the
 * n^3 Lagrangian grid, particle-id order, xyz-interleaved floats in Mpc/h, as written by
 * colapm_get_displacement) to a correction dPsi, and is trained on pairs of runs from the same
 * seeds with targets dPsi = Psi_fine - Psi_coarse. Plain COLA stays the fallback: without the
 * correction nothing changes.
 *
 * Network: four periodic (circular-padded) 3x3x3 convolutions, 3 -> 16 -> 16 -> 16 -> 3, with
 * ReLU after the first three; the input is Psi / s_in and the output is scaled by s_out:
 *     dPsi = s_out * net(Psi / s_in).
 * Products are BF16 x BF16 on the tensor cores with FP32 accumulation; activations between
 * layers are stored in BF16; master weights, gradients and the Adam moments are FP32.
 * Loss: mean over all n^3 x 3 values of (net(Psi / s_in) - dPsi_target / s_out)^2.
 *
 * Parameters (COLAPM_NN_PARAMS floats, host arrays): for each layer l = 1..4 with (c_in, c_out)
 * = (3,16), (16,16), (16,16), (16,3): W[27][c_out][c_in] then b[c_out], where the tap index is
 * (dz+1) 9 + (dy+1) 3 + (dx+1) and out[v][o] = b[o] + sum_tap sum_i W[tap][o][i] in[v + d][i]
 * with v + d taken periodically on the n^3 grid ([iz][iy][ix], ix fastest).
 *
 * Conventions as in colapm.h: return COLAPM_OK or a negative COLAPM_E_* code; a network owns its
 * device memory; work runs on the stream given at creation. Field arguments of
 * colapm_nn_forward/grads/train_step are DEVICE pointers to [n^3][3] floats (COLAPM_E_ARG
 * otherwise) that the caller owns and must keep alive until the stream reaches the work.
 */
#ifndef COLAPM_NN_H
#define COLAPM_NN_H

#ifdef __cplusplus
extern "C" {
#endif

#define COLAPM_NN_PARAMS 16467

typedef struct colapm_nn colapm_nn;

typedef struct {
    float s_in, s_out;            /* input and output scales, Mpc/h (> 0)                        */
    float lr, beta1, beta2, eps;  /* Adam (Kingma & Ba 2015) step size and moment constants      */
    int engine;                   /* convolutions: 0 mma.sync (default); 1 tcgen05 tensor cores   */
                                  /* where n % 128 == 0 (mma.sync otherwise)                      */
    unsigned long long seed;      /* He-normal initial weights (splitmix64 + Box-Muller); b = 0  */
} colapm_nn_config;

/* s_in = s_out = 1, lr = 1e-3, beta1 = 0.9, beta2 = 0.999, eps = 1e-8, engine = 0, seed = 1. */
void colapm_nn_default_config(colapm_nn_config* cfg);

/* A network for n^3 fields (n a multiple of 16, 16..1024); allocates about 7 n^3 x 32 bytes of
 * activations plus a few MB. `stream` is a cudaStream_t (may be NULL). Synchronises. */
int colapm_nn_create(int n, const colapm_nn_config* cfg, void* stream, colapm_nn** out);
int colapm_nn_destroy(colapm_nn* nn);

/* Replace or read the FP32 master parameters (host arrays of COLAPM_NN_PARAMS floats). Setting
 * them leaves the Adam moments and step count alone. Both synchronise. */
int colapm_nn_set_params(colapm_nn* nn, const float* params);
int colapm_nn_get_params(colapm_nn* nn, float* params);

/* out = (add ? psi : 0) + s_out * net(psi / s_in); psi and out are distinct device arrays. */
int colapm_nn_forward(colapm_nn* nn, const float* psi, float* out, int add);

/* Forward and backward on one pair without updating: grads (host, COLAPM_NN_PARAMS floats, or
 * NULL) receives dLoss/dparams in the parameter order above, *loss (or NULL) the loss.
 * Synchronises when either output is requested. */
int colapm_nn_grads(colapm_nn* nn, const float* psi, const float* target, float* grads, double* loss);

/* One Adam step on one pair (Psi_coarse, dPsi_target). *loss (or NULL) receives the loss before
 * the update (synchronises when requested). */
int colapm_nn_train_step(colapm_nn* nn, const float* psi, const float* target, double* loss);

/* Adam steps taken; kernels launched by this network so far; wait for its stream (and report
 * COLAPM_E_TIMEOUT if a bounded device-side wait of a tensor-core convolution gave up). */
int colapm_nn_steps(colapm_nn* nn);
long long colapm_nn_launches(colapm_nn* nn);
int colapm_nn_sync(colapm_nn* nn);

#ifdef __cplusplus
}
#endif

#endif /* COLAPM_NN_H */
