// Host side of the surrogate network (include/es_surrogate.h): parameter
// layout, forward pass, loss and backward pass, Adam.  Every arithmetic step
// is a kernel (sur_gemm.cu, sur_kernels.cu).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "../../include/es.h"
#include "../../include/es_surrogate.h"
#include "sur_internal.h"

using namespace es;

struct es_sur {
    es_sur_config cfg;
    int F, H, K, B;  // feature width, hidden, latent, max batch
    long long D;     // outputs per source
    size_t oW1, ob1, oW2, ob2, oW3, ob3, oWd, P;
    cudaStream_t st = nullptr;
    char* pool = nullptr;
    float *p, *g, *m, *v;  // parameters, gradients, Adam moments (FP32)
    __nv_bfloat16* pb;     // BF16 mirror of the parameters (GEMM operands)
    float* scale;          // [4]
    float scale_h[4] = {1.f, 1.f, 1.f, 1.f};  // host copy (GEMM alpha of the fused inference output)
    __nv_bfloat16 *X, *H1b, *H2b, *Zb, *dUb, *dAb, *dH2b, *dH1b;
    __nv_bfloat16 *ZT, *dUT;  // z^T [6K][B] and dU^T [D][B]: K-major operands of dWd = z^T dU
    float *H1, *H2, *A, *U, *dZ, *dA, *dH2, *dH1, *loss, *acc;
    int t = 0;
    // inference copy of the decoder, K-major for the tcgen05 GEMM: WdT [D][6K],
    // rebuilt from the BF16 mirror whenever the parameters changed (ver)
    __nv_bfloat16* WdT = nullptr;
    long long ver = 0, wdt_ver = -1;
};

namespace {

#define CKS(x)                                       \
    do {                                             \
        if ((x) != cudaSuccess) return ES_ERR_CUDA;  \
    } while (0)

bool dev_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int check_batch(const es_sur* s, const void* pos, const void* mt, int B)
{
    if (!s || !pos || !mt || B < 8 || B > s->B || B % 8) return ES_ERR_ARG;
    if (!dev_ptr(pos) || !dev_ptr(mt)) return ES_ERR_ARG;
    return ES_OK;
}

// The K-major copy of the decoder (WdT [D][6K]), rebuilt from the BF16 mirror
// whenever the parameters have changed since (once per Adam step in training).
int ensure_wdt(es_sur* s)
{
    if (!s->WdT && cudaMalloc(&s->WdT, sizeof(__nv_bfloat16) * 6 * s->K * s->D) != cudaSuccess) {
        cudaGetLastError();
        s->WdT = nullptr;
        return ES_ERR_OOM;
    }
    if (s->wdt_ver != s->ver) {
        CKS(transpose_bf16(s->pb + s->oWd, 6LL * s->K, s->D, s->WdT, s->st));
        s->wdt_ver = s->ver;
    }
    return ES_OK;
}

// forward through the decoder on the tcgen05 tensor cores (both operands
// K-major: z [B][6K] and WdT [D][6K]): s->U = z Wd in normalized units, or for
// inference (out != nullptr) one product writing out directly, the columns of
// component c scaled by that component's RMS.
int forward(es_sur* s, const float* pos, const float* mt, int B, float* out = nullptr)
{
    int rc = ensure_wdt(s);
    if (rc != ES_OK) return rc;
    const __nv_bfloat16* W1 = s->pb + s->oW1;
    const __nv_bfloat16* W2 = s->pb + s->oW2;
    const __nv_bfloat16* W3 = s->pb + s->oW3;
    CKS(sur_features(pos, B, s->cfg.nfreq, s->F, s->X, s->st));
    CKS(gemm_bf16(B, s->H, s->F, s->X, s->F, false, W1, s->H, false, s->H1, s->H, 1.f, 0.f, 1, s->st));
    CKS(sur_bias_act(s->H1, s->p + s->ob1, B, s->H, true, s->H1b, s->st));
    CKS(gemm_bf16(B, s->H, s->H, s->H1b, s->H, false, W2, s->H, false, s->H2, s->H, 1.f, 0.f, 1, s->st));
    CKS(sur_bias_act(s->H2, s->p + s->ob2, B, s->H, true, s->H2b, s->st));
    CKS(gemm_bf16(B, s->K, s->H, s->H2b, s->H, false, W3, s->K, false, s->A, s->K, 1.f, 0.f, 1, s->st));
    CKS(sur_bias_act(s->A, s->p + s->ob3, B, s->K, false, nullptr, s->st));
    CKS(sur_outer(mt, s->A, B, s->K, s->Zb, s->st));
    if (out) {
        // one product over all four components, each column block scaled by its component's RMS
        CKS(gemm_bf16_tc(B, (int)s->D, 6 * s->K, s->Zb, 6 * s->K, s->WdT, 6 * s->K, out, (int)s->D, 1.f, 0.f, 1, s->st,
                         s->scale_h, (int)(s->D / 4)));
    } else
        CKS(gemm_bf16(B, (int)s->D, 6 * s->K, s->Zb, 6 * s->K, false, s->WdT, 6 * s->K, true, s->U, (int)s->D, 1.f,
                      0.f, 1, s->st));
    return ES_OK;
}

// gradients into s->g, given s->dUb from the loss
int backward(es_sur* s, const float* mt, int B)
{
    const int K6 = 6 * s->K, D = (int)s->D;
    const __nv_bfloat16* W2 = s->pb + s->oW2;
    const __nv_bfloat16* W3 = s->pb + s->oW3;
    const __nv_bfloat16* Wd = s->pb + s->oWd;
    // decoder: dWd = z^T dU through the K-major transposes (both on tcgen05), dz = dU Wd^T
    // (long K = D: split-K)
    CKS(transpose_bf16(s->Zb, B, K6, s->ZT, s->st));
    CKS(transpose_bf16(s->dUb, B, D, s->dUT, s->st));
    CKS(gemm_bf16(K6, D, B, s->ZT, B, false, s->dUT, B, true, s->g + s->oWd, D, 1.f, 0.f, 1, s->st));
    const int split = (int)std::max<long long>(1, std::min<long long>(256, s->D / 2048));
    CKS(gemm_bf16(B, K6, D, s->dUb, D, false, Wd, D, true, s->dZ, K6, 1.f, 0.f, split, s->st));
    CKS(sur_contract(mt, s->dZ, B, s->K, s->dA, s->dAb, s->st));
    // latent layer
    CKS(sur_colsum(s->dA, B, s->K, s->g + s->ob3, s->st));
    CKS(gemm_bf16(s->H, s->K, B, s->H2b, s->H, true, s->dAb, s->K, false, s->g + s->oW3, s->K, 1.f, 0.f, 1, s->st));
    CKS(gemm_bf16(B, s->H, s->K, s->dAb, s->K, false, W3, s->K, true, s->dH2, s->H, 1.f, 0.f, 1, s->st));
    CKS(sur_relu_grad(s->dH2, s->H2, (size_t)B * s->H, s->dH2b, s->st));
    // hidden 2
    CKS(sur_colsum(s->dH2, B, s->H, s->g + s->ob2, s->st));
    CKS(gemm_bf16(s->H, s->H, B, s->H1b, s->H, true, s->dH2b, s->H, false, s->g + s->oW2, s->H, 1.f, 0.f, 1, s->st));
    CKS(gemm_bf16(B, s->H, s->H, s->dH2b, s->H, false, W2, s->H, true, s->dH1, s->H, 1.f, 0.f, 1, s->st));
    CKS(sur_relu_grad(s->dH1, s->H1, (size_t)B * s->H, s->dH1b, s->st));
    // hidden 1
    CKS(sur_colsum(s->dH1, B, s->H, s->g + s->ob1, s->st));
    CKS(gemm_bf16(s->F, s->H, B, s->X, s->F, true, s->dH1b, s->H, false, s->g + s->oW1, s->H, 1.f, 0.f, 1, s->st));
    return ES_OK;
}

}  // namespace

extern "C" {

int es_sur_create(const es_sur_config* cfg, es_sur** out)
{
    if (!cfg || !out) return ES_ERR_ARG;
    *out = nullptr;
    const es_sur_config& c = *cfg;
    if (c.nfreq < 0 || c.nfreq > 16 || c.hidden < 8 || c.hidden % 8 || c.latent < 8 || c.latent % 8 || c.n_rcv < 1 ||
        c.nt < 8 || c.nt % 8 || c.max_batch < 8 || c.max_batch % 8)
        return ES_ERR_ARG;
    es_sur* s = new (std::nothrow) es_sur();
    if (!s) return ES_ERR_OOM;
    s->cfg = c;
    s->F = (3 + 6 * c.nfreq + 7) / 8 * 8;
    s->H = c.hidden;
    s->K = c.latent;
    s->B = c.max_batch;
    s->D = 4LL * c.n_rcv * c.nt;
    size_t o = 0;
    auto seg = [&](size_t n) { size_t r = o; o += (n + 7) / 8 * 8; return r; };
    s->oW1 = seg((size_t)s->F * s->H);
    s->ob1 = seg(s->H);
    s->oW2 = seg((size_t)s->H * s->H);
    s->ob2 = seg(s->H);
    s->oW3 = seg((size_t)s->H * s->K);
    s->ob3 = seg(s->K);
    s->oWd = seg((size_t)6 * s->K * s->D);
    s->P = o;
    const size_t B = s->B, P = s->P, H = s->H, K = s->K, D = s->D, F = s->F;
    const size_t f32 = 4 * (4 * P + 4 + B * (2 * H + K + D + 6 * K + K + 2 * H + 2) + 128);
    const size_t b16 = 2 * (P + B * (F + 2 * H + 6 * K + D + K + 2 * H) + B * (6 * K + D)) + 2048;
    if (cudaMalloc(&s->pool, f32 + b16) != cudaSuccess) {
        delete s;
        return ES_ERR_OOM;
    }
    float* fp = reinterpret_cast<float*>(s->pool);
    auto takef = [&](size_t n) { float* r = fp; fp += (n + 7) / 8 * 8; return r; };
    s->p = takef(P);
    s->g = takef(P);
    s->m = takef(P);
    s->v = takef(P);
    s->scale = takef(4);
    s->H1 = takef(B * H);
    s->H2 = takef(B * H);
    s->A = takef(B * K);
    s->U = takef(B * D);
    s->dZ = takef(B * 6 * K);
    s->dA = takef(B * K);
    s->dH2 = takef(B * H);
    s->dH1 = takef(B * H);
    s->loss = takef(8);
    s->acc = takef(2 * B);
    __nv_bfloat16* bp = reinterpret_cast<__nv_bfloat16*>(fp);
    auto takeb = [&](size_t n) { __nv_bfloat16* r = bp; bp += (n + 7) / 8 * 8; return r; };
    s->pb = takeb(P);
    s->X = takeb(B * F);
    s->H1b = takeb(B * H);
    s->H2b = takeb(B * H);
    s->Zb = takeb(B * 6 * K);
    s->dUb = takeb(B * D);
    s->dAb = takeb(B * K);
    s->dH2b = takeb(B * H);
    s->dH1b = takeb(B * H);
    s->ZT = takeb(6 * K * B);
    s->dUT = takeb(D * B);
    const float ones[4] = {1.f, 1.f, 1.f, 1.f};
    cudaError_t e = cudaMemcpy(s->scale, ones, sizeof ones, cudaMemcpyHostToDevice);
    // N(0, 1/fan_in) weights, zero biases, decoder scaled so the first outputs are small
    if (e == cudaSuccess) e = cudaMemset(s->p, 0, sizeof(float) * P);
    if (e == cudaSuccess) e = sur_init_normal(s->p + s->oW1, F * H, 1.f / std::sqrt((float)(3 + 6 * c.nfreq)), c.seed + 1, 0);
    if (e == cudaSuccess) e = sur_init_normal(s->p + s->oW2, H * H, std::sqrt(2.f / H), c.seed + 2, 0);
    if (e == cudaSuccess) e = sur_init_normal(s->p + s->oW3, H * K, std::sqrt(1.f / H), c.seed + 3, 0);
    if (e == cudaSuccess) e = sur_init_normal(s->p + s->oWd, 6 * K * D, 0.1f / std::sqrt(6.f * K), c.seed + 4, 0);
    if (e == cudaSuccess) e = cudaMemset(s->m, 0, sizeof(float) * P);
    if (e == cudaSuccess) e = cudaMemset(s->v, 0, sizeof(float) * P);
    if (e == cudaSuccess) e = cast_bf16(s->p, s->pb, P, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        es_sur_destroy(s);
        return ES_ERR_CUDA;
    }
    *out = s;
    return ES_OK;
}

void es_sur_destroy(es_sur* s)
{
    if (!s) return;
    cudaFree(s->WdT);
    cudaFree(s->pool);
    delete s;
}

int es_sur_set_stream(es_sur* s, void* stream)
{
    if (!s) return ES_ERR_ARG;
    s->st = static_cast<cudaStream_t>(stream);
    return ES_OK;
}

long long es_sur_num_params(const es_sur* s) { return s ? (long long)s->P : (long long)ES_ERR_ARG; }

int es_sur_get_params(es_sur* s, float* params)
{
    if (!s || !params) return ES_ERR_ARG;
    CKS(cudaMemcpyAsync(params, s->p, sizeof(float) * s->P, cudaMemcpyDefault, s->st));
    CKS(cudaStreamSynchronize(s->st));
    return ES_OK;
}

int es_sur_set_params(es_sur* s, const float* params)
{
    if (!s || !params) return ES_ERR_ARG;
    CKS(cudaMemcpyAsync(s->p, params, sizeof(float) * s->P, cudaMemcpyDefault, s->st));
    CKS(cast_bf16(s->p, s->pb, s->P, s->st));
    CKS(cudaStreamSynchronize(s->st));
    s->ver += 1;
    return ES_OK;
}

int es_sur_set_output_scale(es_sur* s, const float* scale4)
{
    if (!s || !scale4) return ES_ERR_ARG;
    for (int c = 0; c < 4; ++c)
        if (!(scale4[c] > 0) || !std::isfinite(scale4[c])) return ES_ERR_ARG;
    CKS(cudaMemcpyAsync(s->scale, scale4, 4 * sizeof(float), cudaMemcpyHostToDevice, s->st));
    CKS(cudaStreamSynchronize(s->st));
    for (int c = 0; c < 4; ++c) s->scale_h[c] = scale4[c];
    return ES_OK;
}

int es_sur_fit_output_scale(es_sur* s, const float* targets, int n)
{
    if (!s || !targets || n < 1 || !dev_ptr(targets)) return ES_ERR_ARG;
    cudaGetLastError();
    CKS(sur_comp_sumsq(targets, n, s->D / 4, s->loss, s->st));
    float ss[4];
    CKS(cudaMemcpyAsync(ss, s->loss, sizeof ss, cudaMemcpyDeviceToHost, s->st));
    CKS(cudaStreamSynchronize(s->st));
    float sc[4];
    for (int c = 0; c < 4; ++c) sc[c] = ss[c] > 0 ? std::sqrt(ss[c] / ((double)n * (s->D / 4))) : 1.f;
    return es_sur_set_output_scale(s, sc);
}

int es_sur_predict(es_sur* s, const float* pos, const float* mt, int B, float* out)
{
    int rc = check_batch(s, pos, mt, B);
    if (rc != ES_OK) return rc;
    if (!out || !dev_ptr(out)) return ES_ERR_ARG;
    cudaGetLastError();
    if ((rc = forward(s, pos, mt, B, out)) != ES_OK) return rc;
    return ES_OK;
}

int es_sur_loss_grad(es_sur* s, const float* pos, const float* mt, const float* target, int B, float* loss,
                     float* per_sample, float* grads)
{
    int rc = check_batch(s, pos, mt, B);
    if (rc != ES_OK) return rc;
    if (!target || !dev_ptr(target) || (per_sample && !dev_ptr(per_sample)) || (grads && !dev_ptr(grads)))
        return ES_ERR_ARG;
    cudaGetLastError();
    if ((rc = forward(s, pos, mt, B)) != ES_OK) return rc;
    CKS(sur_loss(s->U, target, s->scale, B, s->D / 4, 1e-30f, grads ? s->dUb : nullptr, s->loss, s->acc, per_sample,
                 s->st));
    if (grads) {
        if ((rc = backward(s, mt, B)) != ES_OK) return rc;
        CKS(cudaMemcpyAsync(grads, s->g, sizeof(float) * s->P, cudaMemcpyDeviceToDevice, s->st));
    }
    if (loss) CKS(cudaMemcpyAsync(loss, s->loss, sizeof(float), cudaMemcpyDeviceToHost, s->st));
    CKS(cudaStreamSynchronize(s->st));
    return ES_OK;
}

int es_sur_train_step(es_sur* s, const float* pos, const float* mt, const float* target, int B, float lr, float* loss)
{
    int rc = check_batch(s, pos, mt, B);
    if (rc != ES_OK) return rc;
    if (!target || !dev_ptr(target) || !(lr > 0)) return ES_ERR_ARG;
    cudaGetLastError();
    if ((rc = forward(s, pos, mt, B)) != ES_OK) return rc;
    CKS(sur_loss(s->U, target, s->scale, B, s->D / 4, 1e-30f, s->dUb, s->loss, s->acc, nullptr, s->st));
    if ((rc = backward(s, mt, B)) != ES_OK) return rc;
    s->t += 1;
    // the MLP's parameters, then the decoder (the last segment) with its K-major copy refreshed
    // in the same pass
    const size_t K6 = 6 * (size_t)s->K;
    CKS(sur_adam(s->p, s->g, s->m, s->v, s->oWd, lr, 0.9f, 0.999f, 1e-8f, s->t, s->pb, s->st));
    CKS(sur_adam_t(s->p + s->oWd, s->g + s->oWd, s->m + s->oWd, s->v + s->oWd, (long long)K6, s->D, lr, 0.9f, 0.999f,
                   1e-8f, s->t, s->pb + s->oWd, s->WdT, s->st));
    s->ver += 1;
    s->wdt_ver = s->ver;
    if (loss) {
        CKS(cudaMemcpyAsync(loss, s->loss, sizeof(float), cudaMemcpyDeviceToHost, s->st));
        CKS(cudaStreamSynchronize(s->st));
    }
    return ES_OK;
}

int es_sur_combine(const float* G, int n_loc, long long D, const int* loc, const float* mt, int B, float* out,
                   void* stream)
{
    if (!G || !loc || !mt || !out || n_loc < 1 || D < 1 || B < 0) return ES_ERR_ARG;
    if (!dev_ptr(G) || !dev_ptr(loc) || !dev_ptr(mt) || !dev_ptr(out)) return ES_ERR_ARG;
    if (B == 0) return ES_OK;
    cudaGetLastError();
    CKS(sur_combine(G, D, loc, mt, B, out, static_cast<cudaStream_t>(stream)));
    return ES_OK;
}

int es_gemm_status(void)
{
    if (cudaDeviceSynchronize() != cudaSuccess) return ES_ERR_CUDA;
    unsigned v = 0;
    if (gemm_tc_status(&v) != cudaSuccess) return ES_ERR_CUDA;
    return v ? ES_ERR_TIMEOUT : ES_OK;
}

int es_gemm_wait_probe(double seconds, void* stream)
{
    if (!(seconds > 0.0) || seconds > 2.0) return ES_ERR_ARG;
    cudaGetLastError();
    CKS(gemm_wait_probe(seconds, static_cast<cudaStream_t>(stream)));
    return ES_OK;
}

int es_gemm_bf16(int M, int N, int K, const void* A, int lda, int a_t, const void* B, int ldb, int b_nk, float* C,
                 int ldc, float alpha, float beta, int split_k, void* stream)
{
    if (M < 0 || N < 0 || K < 0 || !A || !B || !C || K % 8 || lda % 8 || ldb % 8 || (a_t && M % 8) ||
        (!b_nk && N % 8) || (!a_t && lda < K) || (a_t && lda < M) || (b_nk && ldb < K) || (!b_nk && ldb < N) ||
        ldc < N)
        return ES_ERR_ARG;
    if (!dev_ptr(A) || !dev_ptr(B) || !dev_ptr(C)) return ES_ERR_ARG;
    cudaGetLastError();
    CKS(gemm_bf16(M, N, K, static_cast<const __nv_bfloat16*>(A), lda, a_t != 0, static_cast<const __nv_bfloat16*>(B),
                  ldb, b_nk != 0, C, ldc, alpha, beta, split_k, static_cast<cudaStream_t>(stream)));
    return ES_OK;
}

}  // extern "C"
