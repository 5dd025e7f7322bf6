/*
 * es_surrogate.h -- C ABI of the learned surrogate in libes.so: a small
 * network trained on the solver's own 4C traces that maps a point source's
 * position and moment tensor to its seismograms (the "proxy" for the forward
 * simulation that Das, Chen & Hobson name as future work, Sec. VII-C).  The
 * solver (es.h) stays the fallback and the reference for the surrogate's error.
 *
 * Network (BF16 operands, FP32 accumulation, FP32 master weights, Adam):
 *   x = features(position) = [p, sin(2^j pi p), cos(2^j pi p)], j < nfreq,
 *       p = position scaled to [-1, 1]^3, zero padded to a multiple of 8
 *   h1 = relu(x W1 + b1), h2 = relu(h1 W2 + b2), a = h2 W3 + b3  (latent K)
 *   z[c K + k] = M_c a_k            (M = Mxx Myy Mzz Mxy Mxz Myz)
 *   y = (z Wd) * s                  (D = 4 n_rcv nt outputs, [4][n_rcv][nt])
 * so the prediction is exactly linear in the moment tensor, as the elastic
 * equations are (Sec. IV).  s[c] is a fixed per-component output scale
 * (pressure and velocity differ by orders of magnitude).
 * Loss: mean over samples of the squared relative L2 error of the whole 4C
 * seismogram after dividing each component by its scale:
 *   l = sum_c |(y_c - t_c) / s_c|^2 / (sum_c |t_c / s_c|^2 + eps).
 *
 * Parameters, in this order in one FP32 vector: W1 [F][H], b1 [H], W2 [H][H],
 * b2 [H], W3 [H][K], b3 [K], Wd [6K][D] (row-major, F = padded feature width).
 * All array arguments are device pointers unless stated; calls are ordered on
 * the surrogate's stream.  Errors as in es.h (ES_ERR_*).
 */
#ifndef ES_SURROGATE_H
#define ES_SURROGATE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct es_sur es_sur;

typedef struct {
    int nfreq;              /* Fourier frequencies per coordinate */
    int hidden;             /* H, multiple of 8 */
    int latent;             /* K, multiple of 8 */
    int n_rcv, nt;          /* output D = 4 n_rcv nt, nt multiple of 8 */
    int max_batch;          /* largest batch of sources per call */
    unsigned long long seed;/* weight initialisation */
} es_sur_config;

/* Creates the network with initial weights N(0, 1/fan_in) (decoder scaled
 * down), output scales 1, Adam state zero. */
int es_sur_create(const es_sur_config* cfg, es_sur** out);
void es_sur_destroy(es_sur* s);
int es_sur_set_stream(es_sur* s, void* stream);
long long es_sur_num_params(const es_sur* s);
/* params: host or device, es_sur_num_params floats. */
int es_sur_get_params(es_sur* s, float* params);
int es_sur_set_params(es_sur* s, const float* params);
/* Output scale per component (host, 4 floats). */
int es_sur_set_output_scale(es_sur* s, const float* scale4);

/* Sets each component's output scale to the RMS of that component over the
 * n training targets [n][D] (device). */
int es_sur_fit_output_scale(es_sur* s, const float* targets, int n);

/* Prediction for B sources: pos [B][3] in [-1, 1], mt [B][6]; out [B][D]. */
int es_sur_predict(es_sur* s, const float* pos, const float* mt, int B, float* out);

/* Loss (host float) and, when grads != NULL, the gradient of the loss with
 * respect to every parameter (device, es_sur_num_params floats), for the
 * targets [B][D]; per_sample (device [B] or NULL) gets each sample's l. */
int es_sur_loss_grad(es_sur* s, const float* pos, const float* mt, const float* target, int B, float* loss,
                     float* per_sample, float* grads);

/* One Adam step (lr, beta1 0.9, beta2 0.999, eps 1e-8) on the batch; loss
 * (host, optional) receives the batch loss before the step. */
int es_sur_train_step(es_sur* s, const float* pos, const float* mt, const float* target, int B, float lr,
                      float* loss);

/* Seismograms of (location, moment tensor) pairs from a catalog of unit
 * responses, by the exact linearity of the elastic equations (Sec. IV):
 * out[b] = sum_c mt[b][c] G[loc[b]][c], with G [n_loc][6][D] the solver's
 * traces for the six unit moment tensors (Mxx Myy Mzz Mxy Mxz Myz) at each
 * location.  Device arrays; loc values must lie in [0, n_loc) (not checked on
 * the device). */
int es_sur_combine(const float* G, int n_loc, long long D, const int* loc, const float* mt, int B, float* out,
                   void* stream);

/* The network's GEMM, exposed for testing and reuse:
 * C[M][N] = alpha op(A) op(B) + beta C with BF16 A, B (bf16 bit patterns) and
 * FP32 C, all device memory.  A is row-major [M][K] (lda), or stored [K][M]
 * when a_t; B is stored [N][K] when b_nk, else [K][N].  K, lda, ldb multiples
 * of 8 (and M when a_t, N when !b_nk).  split_k > 1 splits K across CTAs
 * (atomic FP32 adds: summation order not fixed).  FP32 accumulation.
 * Both operands K-major (a_t == 0, b_nk != 0; A and B 16-byte aligned): the
 * fifth-generation tensor cores -- TMA-fed 4-stage shared-memory ring,
 * tcgen05.mma 128 x 256 x 16 into a tensor-memory accumulator, 128 x 256
 * tiles.  Other storage orders: mma.sync m16n8k16 with ldmatrix operands.
 * Device waits in the tcgen05 kernel are bounded; see es_gemm_status. */
int es_gemm_bf16(int M, int N, int K, const void* A, int lda, int a_t, const void* B, int ldb, int b_nk, float* C,
                 int ldc, float alpha, float beta, int split_k, void* stream);

/* Synchronizes the device, then reports and clears the tcgen05 GEMM's
 * device status word: ES_OK, or ES_ERR_TIMEOUT if any of its bounded
 * mbarrier waits ran out since the last call (that launch's C is undefined). */
int es_gemm_status(void);

/* Test hook for the failure path of those waits (no fault, no hang): launches
 * on `stream` one kernel in which a single thread waits, through the same
 * bounded wait as the tcgen05 GEMM, on a barrier phase that nothing completes;
 * after `seconds` of device time (0 < seconds <= 2) it gives up, sets the
 * status word and returns, so the next es_gemm_status() reports
 * ES_ERR_TIMEOUT and the context stays usable.  Returns ES_OK, ES_ERR_ARG
 * (seconds out of range) or ES_ERR_CUDA. */
int es_gemm_wait_probe(double seconds, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* ES_SURROGATE_H */
