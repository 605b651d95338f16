// Parameter selection for M-HDC: features, a small MLP (forward, backward and
// Adam in hand-written kernels), the exhaustive autotuner and mhdc_select.
//
// The paper fixes theta = 0.6 and a block width after a sweep (Sec. 6.4.3) and
// leaves "whether M-HDC should be used" as future work (Sec. 7); its
// performance model (Sec. 5.3, Eq. 11) estimates the gain from alpha and beta.
// Here the choice of (n_b, theta, value dtype) is a regression: the MLP maps
// per-block diagonal-occupancy histograms to the (log, relative) time of
// every candidate of a fixed grid, trained on times this library measures.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "mhdc_internal.cuh"

namespace mhdc {
namespace {

constexpr int FEAT_NB[3] = {256, 1024, 4096};
constexpr int CAND_NB[5] = {512, 1024, 2048, 4096, 8192};
constexpr double CAND_THETA[3] = {0.5, 0.6, 0.8};
constexpr int CAND_DT[3] = {MHDC_F64, MHDC_F32, MHDC_BF16};

// ---------------------------------------------------------------- MLP kernels

// Z = X W^T + b;  Y = relu(Z) if relu else Z.   X [B x I], W [O x I].
__global__ void k_lin_fwd(int B, int I, int O, const float *__restrict__ X,
                          const float *__restrict__ W, const float *__restrict__ bias,
                          float *__restrict__ Z, float *__restrict__ Y, int relu)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)B * O) return;
    const int b = (int)(t / O), o = (int)(t % O);
    float z = bias[o];
    const float *x = X + (int64_t)b * I;
    const float *w = W + (int64_t)o * I;
    for (int i = 0; i < I; i++) z = fmaf(x[i], w[i], z);
    Z[t] = z;
    Y[t] = relu ? fmaxf(z, 0.f) : z;
}

// dX[b][i] = sum_o dZ[b][o] W[o][i], times relu'(Zprev[b][i]) when Zprev != NULL.
__global__ void k_lin_bwd_x(int B, int I, int O, const float *__restrict__ dZ,
                            const float *__restrict__ W, const float *__restrict__ Zprev,
                            float *__restrict__ dX)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)B * I) return;
    const int b = (int)(t / I), i = (int)(t % I);
    float s = 0.f;
    const float *dz = dZ + (int64_t)b * O;
    for (int o = 0; o < O; o++) s = fmaf(dz[o], W[(int64_t)o * I + i], s);
    if (Zprev && Zprev[t] <= 0.f) s = 0.f;
    dX[t] = s;
}

// dW[o][i] = sum_b dZ[b][o] X[b][i];  db[o] = sum_b dZ[b][o]  (i == I: the bias).
__global__ void k_lin_bwd_w(int B, int I, int O, const float *__restrict__ dZ,
                            const float *__restrict__ X, float *__restrict__ dW,
                            float *__restrict__ db)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)O * (I + 1)) return;
    const int o = (int)(t / (I + 1)), i = (int)(t % (I + 1));
    float s = 0.f;
    for (int b = 0; b < B; b++)
        s = fmaf(dZ[(int64_t)b * O + o], i < I ? X[(int64_t)b * I + i] : 1.f, s);
    if (i < I) dW[(int64_t)o * I + i] = s;
    else db[o] = s;
}

// Masked mean squared error: L = sum M (Y - T)^2 / sum M;  dY = 2 M (Y - T) / sum M.
// One CTA; also writes L to *loss.
__global__ void k_mse(int n, const float *__restrict__ Y, const float *__restrict__ T,
                      const float *__restrict__ M, float *__restrict__ dY, float *__restrict__ loss)
{
    __shared__ float red[2][256];
    float cnt = 0.f, sq = 0.f;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        cnt += M[k];
        const float d = Y[k] - T[k];
        sq += M[k] * d * d;
    }
    red[0][threadIdx.x] = cnt;
    red[1][threadIdx.x] = sq;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            red[0][threadIdx.x] += red[0][threadIdx.x + s];
            red[1][threadIdx.x] += red[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    const float inv = red[0][0] > 0.f ? 1.f / red[0][0] : 0.f;
    for (int k = threadIdx.x; k < n; k += blockDim.x) dY[k] = 2.f * M[k] * (Y[k] - T[k]) * inv;
    if (threadIdx.x == 0) *loss = red[1][0] * inv;
}

// Adam (Kingma & Ba 2015), bias-corrected with c1 = 1 - b1^t, c2 = 1 - b2^t.
__global__ void k_adam(int64_t P, float *__restrict__ p, const float *__restrict__ g,
                       float *__restrict__ m, float *__restrict__ v, float lr, float b1, float b2,
                       float eps, float c1, float c2)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P) return;
    m[k] = b1 * m[k] + (1.f - b1) * g[k];
    v[k] = b2 * v[k] + (1.f - b2) * g[k] * g[k];
    p[k] -= lr * (m[k] / c1) / (sqrtf(v[k] / c2) + eps);
}

inline unsigned grid_of(int64_t m) { return (unsigned)((m + 255) / 256); }

uint64_t splitmix(uint64_t &s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace
}  // namespace mhdc

using namespace mhdc;

// Layer sizes: F -> H -> H -> O; parameters W1 [H x F], b1 [H], W2 [H x H],
// b2 [H], W3 [O x H], b3 [O], contiguous in that order.
struct mhdc_mlp {
    int F = 0, H = 0, O = 0;
    int64_t P = 0;
    float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    int64_t step = 0;
    float *work = nullptr;  // activations of the last forward (training)
    int work_batch = 0;
    float *loss = nullptr;
};

namespace {

int64_t mlp_param_count(int F, int H, int O)
{
    return (int64_t)H * F + H + (int64_t)H * H + H + (int64_t)O * H + O;
}

struct Views {
    float *W1, *b1, *W2, *b2, *W3, *b3;
};

Views views(const mhdc_mlp *M, float *base)
{
    Views v;
    v.W1 = base;
    v.b1 = v.W1 + (int64_t)M->H * M->F;
    v.W2 = v.b1 + M->H;
    v.b2 = v.W2 + (int64_t)M->H * M->H;
    v.W3 = v.b2 + M->H;
    v.b3 = v.W3 + (int64_t)M->O * M->H;
    return v;
}

// work layout for batch B: Z1, A1, Z2, A2 [B x H], Y [B x O], dY [B x O],
// dA2 [B x H], dA1 [B x H]
int ensure_work(mhdc_mlp *M, int B)
{
    if (M->work && M->work_batch >= B) return MHDC_OK;
    dfree(M->work);
    M->work = nullptr;
    const int64_t words = (int64_t)B * (6 * M->H + 2 * M->O);
    MHDC_CUDA_TRY(dmalloc((void **)&M->work, sizeof(float) * (size_t)words));
    M->work_batch = B;
    return MHDC_OK;
}

int forward(mhdc_mlp *M, int B, const float *X, float *Yout, cudaStream_t st)
{
    const Views p = views(M, M->params);
    float *Z1 = M->work, *A1 = Z1 + (int64_t)B * M->H, *Z2 = A1 + (int64_t)B * M->H,
          *A2 = Z2 + (int64_t)B * M->H, *Y = A2 + (int64_t)B * M->H;
    k_lin_fwd<<<grid_of((int64_t)B * M->H), 256, 0, st>>>(B, M->F, M->H, X, p.W1, p.b1, Z1, A1, 1);
    k_lin_fwd<<<grid_of((int64_t)B * M->H), 256, 0, st>>>(B, M->H, M->H, A1, p.W2, p.b2, Z2, A2, 1);
    k_lin_fwd<<<grid_of((int64_t)B * M->O), 256, 0, st>>>(B, M->H, M->O, A2, p.W3, p.b3, Y, Y, 0);
    MHDC_LAUNCH_CHECK("k_lin_fwd");
    if (Yout && Yout != Y)
        MHDC_CUDA_TRY(cudaMemcpyAsync(Yout, Y, sizeof(float) * (size_t)B * M->O,
                                      cudaMemcpyDeviceToDevice, st));
    return MHDC_OK;
}

// forward + masked MSE + backward into M->grads
int gradient(mhdc_mlp *M, int B, const float *X, const float *T, const float *Mask,
             cudaStream_t st)
{
    int rc = ensure_work(M, B);
    if (rc != MHDC_OK) return rc;
    rc = forward(M, B, X, nullptr, st);
    if (rc != MHDC_OK) return rc;
    const Views p = views(M, M->params), g = views(M, M->grads);
    float *Z1 = M->work, *A1 = Z1 + (int64_t)B * M->H, *Z2 = A1 + (int64_t)B * M->H,
          *A2 = Z2 + (int64_t)B * M->H, *Y = A2 + (int64_t)B * M->H,
          *dY = Y + (int64_t)B * M->O, *dA2 = dY + (int64_t)B * M->O, *dA1 = dA2 + (int64_t)B * M->H;
    k_mse<<<1, 256, 0, st>>>(B * M->O, Y, T, Mask, dY, M->loss);
    k_lin_bwd_w<<<grid_of((int64_t)M->O * (M->H + 1)), 256, 0, st>>>(B, M->H, M->O, dY, A2, g.W3, g.b3);
    k_lin_bwd_x<<<grid_of((int64_t)B * M->H), 256, 0, st>>>(B, M->H, M->O, dY, p.W3, Z2, dA2);
    k_lin_bwd_w<<<grid_of((int64_t)M->H * (M->H + 1)), 256, 0, st>>>(B, M->H, M->H, dA2, A1, g.W2, g.b2);
    k_lin_bwd_x<<<grid_of((int64_t)B * M->H), 256, 0, st>>>(B, M->H, M->H, dA2, p.W2, Z1, dA1);
    k_lin_bwd_w<<<grid_of((int64_t)M->H * (M->F + 1)), 256, 0, st>>>(B, M->F, M->H, dA1, X, g.W1, g.b1);
    MHDC_LAUNCH_CHECK("mlp backward");
    return MHDC_OK;
}

// ---------------------------------------------------------------- features

int compute_features(int64_t n, const int32_t *rp, const int32_t *col, cudaStream_t st, float *f)
{
    int32_t nnz = 0;
    MHDC_CUDA_TRY(cudaMemcpyAsync(&nnz, rp + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MHDC_CUDA_TRY(cudaStreamSynchronize(st));
    const double dn = (double)(n > 0 ? n : 1), dz = (double)(nnz > 0 ? nnz : 1);
    int k = 0;
    for (int s = 0; s < 3; s++) {
        unsigned long long ent[10], dia[10];
        int rc = feature_hist(n, rp, col, FEAT_NB[s], st, ent, dia);
        if (rc != MHDC_OK) return rc;
        const double nblocks = std::ceil(dn / FEAT_NB[s]);
        for (int b = 0; b < 10; b++) f[k++] = (float)((double)ent[b] / dz);
        for (int b = 0; b < 10; b++) f[k++] = (float)(std::log1p((double)dia[b] / nblocks) / 8.0);
    }
    f[k++] = (float)(std::log2(1.0 + dz / dn) / 6.0);
    f[k++] = (float)(std::log2(dn) / 24.0);
    f[k++] = (float)(std::log2(1.0 + dz) / 32.0);
    f[k++] = 1.0f;
    return MHDC_OK;
}

// Worst-case per-row error bound (relative to sum |a||x|) of a dtype for rows
// of c terms: storage rounding of a and x, then c + 1 accumulations.
double dtype_bound(int dt, double c)
{
    if (dt == MHDC_F64) return 1e-12;
    const double ua = std::ldexp(1.0, -24);
    const double us = dt == MHDC_F32 ? ua : (1 + ua) * (1 + std::ldexp(1.0, -8)) - 1;
    const double k = c + 1;
    const double g = k * ua / (1 - k * ua);
    return (1 + us) * (1 + us) * (1 + g) - 1;
}

// The paper's model (Sec. 5.3.3, Eq. 11 with v_x = 1) generalised to the
// value size s_v: bytes of M-HDC relative to FP64 CSR; alpha and beta of a
// candidate come from the occupancy histogram at its block size.
double model_bytes(const float *f, int s, double theta, int dt, double c)
{
    // entries kept in DIA: bins >= theta; diagonals kept: dia bins >= theta
    double kept = 0.0, diags = 0.0;
    for (int b = (int)std::floor(theta * 10 + 1e-9); b < 10; b++) {
        kept += f[s * 20 + b];
        diags += std::expm1(8.0 * f[s * 20 + 10 + b]);  // diagonals per block
    }
    const double beta = 1.0 - kept;
    const double sv = dt == MHDC_F64 ? 8 : dt == MHDC_F32 ? 4 : 2;
    // per row: dia values, remainder (value + index), row pointer, x, y
    return sv * diags + (sv + 4) * beta * c + 4 + sv + (dt == MHDC_F64 ? 8 : 4);
}

}  // namespace

extern "C" {

int mhdc_num_candidates(void) { return MHDC_NUM_CANDIDATES; }

int mhdc_candidate(int32_t idx, mhdc_params *out)
{
    if (idx < 0 || idx >= MHDC_NUM_CANDIDATES || !out) {
        set_error_msg("mhdc_candidate: index out of range");
        return MHDC_ERR_INVALID_ARG;
    }
    out->dtype = CAND_DT[idx / 15];
    out->n_b = CAND_NB[(idx % 15) / 3];
    out->theta = CAND_THETA[idx % 3];
    out->variant = -1;
    return MHDC_OK;
}

int mhdc_features(int64_t n, const int32_t *d_row_ptr, const int32_t *d_col, void *stream,
                  float *h_features)
{
    if (n < 1 || !d_row_ptr || !h_features) {
        set_error_msg("mhdc_features: invalid argument");
        return MHDC_ERR_INVALID_ARG;
    }
    return compute_features(n, d_row_ptr, d_col, (cudaStream_t)stream, h_features);
}

int mhdc_autotune(int64_t n, const int32_t *d_row_ptr, const int32_t *d_col, const double *d_val,
                  int32_t reps, void *stream, float *h_times_us)
{
    if (n < 1 || !d_row_ptr || !h_times_us || reps < 1) {
        set_error_msg("mhdc_autotune: invalid argument");
        return MHDC_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    void *x = nullptr, *y = nullptr;
    MHDC_CUDA_TRY(dmalloc(&x, 8 * (size_t)n));
    cudaError_t e = dmalloc(&y, 8 * (size_t)n);
    if (e != cudaSuccess) {
        dfree(x);
        set_error("cudaMalloc", e);
        return cuda_status(e);
    }
    cudaMemsetAsync(x, 0, 8 * (size_t)n, st);  // x = 0 (any x gives the same time)
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = MHDC_OK;
    for (int c = 0; c < MHDC_NUM_CANDIDATES && rc == MHDC_OK; c++) {
        mhdc_params p;
        mhdc_candidate(c, &p);
        mhdc_matrix *A = nullptr;
        rc = build_matrix(n, d_row_ptr, d_col, d_val, p.n_b, p.theta, p.dtype, MHDC_MODE_BLOCK, st, &A);
        if (rc != MHDC_OK) {
            h_times_us[c] = -1.f;  // could not be built (e.g. out of memory): excluded
            if (rc == MHDC_ERR_OOM) rc = MHDC_OK;
            continue;
        }
        for (int r = 0; r < 2 && rc == MHDC_OK; r++) rc = launch_spmv(A, x, y, st);
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps && rc == MHDC_OK; r++) rc = launch_spmv(A, x, y, st);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        h_times_us[c] = ms * 1000.f / reps;
        free_matrix(A);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dfree(x);
    dfree(y);
    return rc;
}

int mhdc_mlp_create(int32_t n_in, int32_t n_hidden, int32_t n_out, uint64_t seed,
                    mhdc_mlp_handle *out)
{
    if (n_in < 1 || n_hidden < 1 || n_out < 1 || !out) {
        set_error_msg("mhdc_mlp_create: invalid argument");
        return MHDC_ERR_INVALID_ARG;
    }
    mhdc_mlp *M = new mhdc_mlp();
    M->F = n_in;
    M->H = n_hidden;
    M->O = n_out;
    M->P = mlp_param_count(n_in, n_hidden, n_out);
    std::vector<float> h((size_t)M->P);
    // He-uniform weights (limit sqrt(6 / fan_in)), zero biases
    uint64_t s = seed;
    Views v = views(M, h.data());
    auto fill = [&](float *w, int64_t count, int fan_in) {
        const double lim = std::sqrt(6.0 / fan_in);
        for (int64_t k = 0; k < count; k++)
            w[k] = (float)(lim * (2.0 * ((splitmix(s) >> 11) * 0x1.0p-53) - 1.0));
    };
    std::fill(h.begin(), h.end(), 0.f);
    fill(v.W1, (int64_t)M->H * M->F, M->F);
    fill(v.W2, (int64_t)M->H * M->H, M->H);
    fill(v.W3, (int64_t)M->O * M->H, M->H);
    const size_t bytes = sizeof(float) * (size_t)M->P;
    cudaError_t e = dmalloc((void **)&M->params, bytes);
    if (e == cudaSuccess) e = dmalloc((void **)&M->grads, bytes);
    if (e == cudaSuccess) e = dmalloc((void **)&M->m, bytes);
    if (e == cudaSuccess) e = dmalloc((void **)&M->v, bytes);
    if (e == cudaSuccess) e = dmalloc((void **)&M->loss, sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(M->params, h.data(), bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(M->m, 0, bytes);
    if (e == cudaSuccess) e = cudaMemset(M->v, 0, bytes);
    if (e == cudaSuccess) e = cudaMemset(M->grads, 0, bytes);
    if (e != cudaSuccess) {
        set_error("mhdc_mlp_create", e);
        mhdc_mlp_destroy(M);
        return cuda_status(e);
    }
    *out = M;
    return MHDC_OK;
}

int64_t mhdc_mlp_num_params(mhdc_mlp_handle M) { return M ? M->P : -1; }

int mhdc_mlp_get_params(mhdc_mlp_handle M, float *h_params)
{
    if (!M || !h_params) return MHDC_ERR_INVALID_ARG;
    MHDC_CUDA_TRY(cudaMemcpy(h_params, M->params, sizeof(float) * (size_t)M->P,
                             cudaMemcpyDeviceToHost));
    return MHDC_OK;
}

int mhdc_mlp_set_params(mhdc_mlp_handle M, const float *h_params)
{
    if (!M || !h_params) return MHDC_ERR_INVALID_ARG;
    MHDC_CUDA_TRY(cudaMemcpy(M->params, h_params, sizeof(float) * (size_t)M->P,
                             cudaMemcpyHostToDevice));
    M->step = 0;
    MHDC_CUDA_TRY(cudaMemset(M->m, 0, sizeof(float) * (size_t)M->P));
    MHDC_CUDA_TRY(cudaMemset(M->v, 0, sizeof(float) * (size_t)M->P));
    return MHDC_OK;
}

int mhdc_mlp_forward(mhdc_mlp_handle M, int32_t batch, const float *d_X, float *d_Y, void *stream)
{
    if (!M || batch < 1 || !d_X || !d_Y) {
        set_error_msg("mhdc_mlp_forward: invalid argument");
        return MHDC_ERR_INVALID_ARG;
    }
    int rc = ensure_work(M, batch);
    if (rc != MHDC_OK) return rc;
    return forward(M, batch, d_X, d_Y, (cudaStream_t)stream);
}

int mhdc_mlp_grad(mhdc_mlp_handle M, int32_t batch, const float *d_X, const float *d_T,
                  const float *d_M, float *h_grads, float *h_loss, void *stream)
{
    if (!M || batch < 1 || !d_X || !d_T || !d_M) {
        set_error_msg("mhdc_mlp_grad: invalid argument");
        return MHDC_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int rc = gradient(M, batch, d_X, d_T, d_M, st);
    if (rc != MHDC_OK) return rc;
    if (h_grads)
        MHDC_CUDA_TRY(cudaMemcpyAsync(h_grads, M->grads, sizeof(float) * (size_t)M->P,
                                      cudaMemcpyDeviceToHost, st));
    if (h_loss) MHDC_CUDA_TRY(cudaMemcpyAsync(h_loss, M->loss, sizeof(float), cudaMemcpyDeviceToHost, st));
    MHDC_CUDA_TRY(cudaStreamSynchronize(st));
    return MHDC_OK;
}

int mhdc_mlp_train_step(mhdc_mlp_handle M, int32_t batch, const float *d_X, const float *d_T,
                        const float *d_M, float lr, void *stream, float *h_loss)
{
    if (!M || batch < 1 || !d_X || !d_T || !d_M || !(lr > 0.f)) {
        set_error_msg("mhdc_mlp_train_step: invalid argument");
        return MHDC_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int rc = gradient(M, batch, d_X, d_T, d_M, st);
    if (rc != MHDC_OK) return rc;
    M->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)M->step), c2 = 1.f - std::pow(b2, (float)M->step);
    k_adam<<<grid_of(M->P), 256, 0, st>>>(M->P, M->params, M->grads, M->m, M->v, lr, b1, b2, 1e-8f,
                                          c1, c2);
    MHDC_LAUNCH_CHECK("k_adam");
    if (h_loss) {
        MHDC_CUDA_TRY(cudaMemcpyAsync(h_loss, M->loss, sizeof(float), cudaMemcpyDeviceToHost, st));
        MHDC_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return MHDC_OK;
}

int mhdc_mlp_destroy(mhdc_mlp_handle M)
{
    if (!M) return MHDC_OK;
    dfree(M->params);
    dfree(M->grads);
    dfree(M->m);
    dfree(M->v);
    dfree(M->work);
    dfree(M->loss);
    delete M;
    return MHDC_OK;
}

int mhdc_select(int64_t n, const int32_t *d_row_ptr, const int32_t *d_col, const double *d_val,
                double tol, int32_t flags, mhdc_mlp_handle mlp, void *stream, mhdc_params *out)
{
    if (n < 1 || !d_row_ptr || !out || !(tol > 0)) {
        set_error_msg("mhdc_select: invalid argument");
        return MHDC_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int32_t nnz = 0;
    MHDC_CUDA_TRY(cudaMemcpyAsync(&nnz, d_row_ptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MHDC_CUDA_TRY(cudaStreamSynchronize(st));
    const double c = (double)nnz / (double)n;
    bool allowed[3];
    for (int d = 0; d < 3; d++) allowed[d] = d == 0 || dtype_bound(CAND_DT[d], c) <= tol;
    auto ok = [&](int idx) { return allowed[idx / 15]; };
    int best = -1;
    if (flags & MHDC_SELECT_AUTOTUNE) {
        float t[MHDC_NUM_CANDIDATES];
        int rc = mhdc_autotune(n, d_row_ptr, d_col, d_val, 10, stream, t);
        if (rc != MHDC_OK) return rc;
        for (int k = 0; k < MHDC_NUM_CANDIDATES; k++)
            if (ok(k) && t[k] > 0 && (best < 0 || t[k] < t[best])) best = k;
    } else if (flags & MHDC_SELECT_MLP) {
        if (!mlp || mlp->F != MHDC_NUM_FEATURES || mlp->O != MHDC_NUM_CANDIDATES) {
            set_error_msg("mhdc_select: the MLP must map MHDC_NUM_FEATURES to MHDC_NUM_CANDIDATES");
            return MHDC_ERR_INVALID_ARG;
        }
        float f[MHDC_NUM_FEATURES], pred[MHDC_NUM_CANDIDATES];
        int rc = compute_features(n, d_row_ptr, d_col, st, f);
        if (rc != MHDC_OK) return rc;
        float *d = nullptr;
        MHDC_CUDA_TRY(dmalloc((void **)&d, sizeof(float) * (MHDC_NUM_FEATURES + MHDC_NUM_CANDIDATES)));
        cudaMemcpyAsync(d, f, sizeof f, cudaMemcpyHostToDevice, st);
        rc = mhdc_mlp_forward(mlp, 1, d, d + MHDC_NUM_FEATURES, stream);
        if (rc == MHDC_OK)
            cudaMemcpyAsync(pred, d + MHDC_NUM_FEATURES, sizeof pred, cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        dfree(d);
        if (rc != MHDC_OK) return rc;
        for (int k = 0; k < MHDC_NUM_CANDIDATES; k++)
            if (ok(k) && (best < 0 || pred[k] < pred[best])) best = k;
    } else if (flags & MHDC_SELECT_MODEL) {
        float f[MHDC_NUM_FEATURES];
        int rc = compute_features(n, d_row_ptr, d_col, st, f);
        if (rc != MHDC_OK) return rc;
        double bv = 0.0;
        for (int k = 0; k < MHDC_NUM_CANDIDATES; k++) {
            if (!ok(k)) continue;
            mhdc_params p;
            mhdc_candidate(k, &p);
            // nearest feature block size to the candidate's
            const int s = p.n_b <= 512 ? 0 : p.n_b <= 2048 ? 1 : 2;
            const double v = model_bytes(f, s, p.theta, p.dtype, c);
            if (best < 0 || v < bv) {
                best = k;
                bv = v;
            }
        }
    } else {
        // the paper's policy (Sec. 6.4.3): theta = 0.6 and a fixed block width
        // (here 4096 rows), in the cheapest dtype the tolerance allows
        out->n_b = 4096;
        out->theta = 0.6;
        out->dtype = allowed[2] ? MHDC_BF16 : allowed[1] ? MHDC_F32 : MHDC_F64;
        out->variant = -1;
        return MHDC_OK;
    }
    if (best < 0) {
        set_error_msg("mhdc_select: no candidate could be evaluated");
        return MHDC_ERR_UNSUPPORTED;
    }
    return mhdc_candidate(best, out);
}

}  // extern "C"
