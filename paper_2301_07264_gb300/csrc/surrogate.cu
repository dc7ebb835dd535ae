// Learned surrogate of the success probability: a 33 -> 256 -> 256 -> 1 MLP
// trained on the GPU on pass flags produced by the trajectory simulator, and
// the surrogate-bracketed tolerable-rate search (Sec. IV-D, Monte Carlo
// branch: the surrogate proposes the bracket, plain trajectories verify it).
//
// Weights are bfloat16 (with FP32 masters for Adam); every product
// accumulates in FP32. The MLP costs ~1.5e5 FMA per row, negligible next to
// the trajectories that label it, so the kernels are plain tiled SIMT GEMMs.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>

#include "kernels.h"
#include "prof.h"

namespace arso {

constexpr int IN = ARSO_SURROGATE_INPUTS, HID = 256;
constexpr size_t OFF_W1 = 0, OFF_B1 = OFF_W1 + IN * HID, OFF_W2 = OFF_B1 + HID, OFF_B2 = OFF_W2 + HID * HID,
                 OFF_W3 = OFF_B2 + HID, OFF_B3 = OFF_W3 + HID, N_PARAMS = OFF_B3 + 1;
static_assert(N_PARAMS == ARSO_SURROGATE_PARAMS, "parameter layout");

// ------------------------------------------------------------------ GEMM ---
// C[m, n] = epi( sum_k A(m, k) B(k, n) ), A(m, k) = A[m * sam + k * sak],
// B(k, n) = B[k * sbk + n * sbn]; epilogue: + bias[n], relu, or * (mask > 0).
enum { EPI_NONE = 0, EPI_BIAS_RELU = 1, EPI_BIAS = 2, EPI_RELU_MASK = 3 };

__device__ __forceinline__ float ldf(const float *p) { return *p; }
__device__ __forceinline__ float ldf(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

template <typename TA, typename TB>
__global__ void gemm_kernel(int M, int N, int K, const TA *__restrict__ A, long sam, long sak, const TB *__restrict__ B,
                            long sbk, long sbn, float *__restrict__ C, int epi, const TB *__restrict__ bias,
                            const float *__restrict__ mask) {
    __shared__ float As[16][17], Bs[16][17];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int m = blockIdx.y * 16 + ty, n = blockIdx.x * 16 + tx;
    float acc = 0.f;
    for (int k0 = 0; k0 < K; k0 += 16) {
        const int ka = k0 + tx, kb = k0 + ty;
        As[ty][tx] = (m < M && ka < K) ? ldf(A + (long)m * sam + (long)ka * sak) : 0.f;
        Bs[ty][tx] = (kb < K && n < N) ? ldf(B + (long)kb * sbk + (long)n * sbn) : 0.f;
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) acc = fmaf(As[ty][kk], Bs[kk][tx], acc);
        __syncthreads();
    }
    if (m < M && n < N) {
        if (epi == EPI_BIAS_RELU) acc = fmaxf(acc + ldf(bias + n), 0.f);
        else if (epi == EPI_BIAS) acc += ldf(bias + n);
        else if (epi == EPI_RELU_MASK) acc = mask[(long)m * N + n] > 0.f ? acc : 0.f;
        C[(long)m * N + n] = acc;
    }
}

template <typename TA, typename TB>
static void gemm(int M, int N, int K, const TA *A, long sam, long sak, const TB *B, long sbk, long sbn, float *C, int epi,
                 const TB *bias, const float *mask, cudaStream_t st) {
    dim3 block(16, 16), grid((N + 15) / 16, (M + 15) / 16);
    gemm_kernel<TA, TB><<<grid, block, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, epi, bias, mask);
    ARSO_CUDA(cudaGetLastError());
}

// column sums: out[n] = sum_m X[m, n] (bias gradients)
__global__ void colsum_kernel(const float *__restrict__ X, int M, int N, float *out) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int m = 0; m < M; ++m) s += X[(long)m * N + n];
    out[n] = s;
}

// gather and standardise a batch: xb[i, c] = (x[idx[i], c] - mean[c]) / sd[c]
__global__ void gather_norm_kernel(const float *__restrict__ x, const uint32_t *__restrict__ idx, uint64_t base,
                                   int rows, const float *__restrict__ norm, float *xb) {
    const int i = blockIdx.x, c = threadIdx.x;
    if (i >= rows || c >= IN) return;
    const uint64_t r = idx ? idx[base + i] : base + i;
    xb[(long)i * IN + c] = (x[r * IN + c] - norm[c]) / norm[IN + c];
}

// logit gradient of the mean BCE: dz = (sigmoid(z) - y) / B; loss += softplus(z) - y z
__global__ void bce_kernel(const float *__restrict__ z, const float *__restrict__ y, const uint32_t *__restrict__ idx,
                           uint64_t base, int rows, float inv_b, float *dz, double *loss_sum) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (i < rows) {
        const uint64_t r = idx ? idx[base + i] : base + i;
        const float zi = z[i], yi = y[r];
        const float s = 1.f / (1.f + __expf(-zi));
        dz[i] = (s - yi) * inv_b;
        l = (double)(fmaxf(zi, 0.f) + log1pf(__expf(-fabsf(zi))) - yi * zi);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0 && l != 0.0) atomicAdd(loss_sum, l);
}

__global__ void sigmoid_kernel(const float *__restrict__ z, int n, float *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = 1.f / (1.f + __expf(-z[i]));
}

// Adam (Kingma & Ba 2015) on the FP32 masters; refresh the bfloat16 copies
__global__ void adam_kernel(float *w, __nv_bfloat16 *w16, const float *__restrict__ g, float *m, float *v, size_t n,
                            float lr, float b1, float b2, float eps, float c1, float c2) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        w16[i] = __float2bfloat16_rn(wi);
    }
}

__global__ void to_bf16_kernel(const float *__restrict__ w, __nv_bfloat16 *w16, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        w16[i] = __float2bfloat16_rn(w[i]);
}

// per-column sum and sum of squares (FP64) for the standardisation
__global__ void moments_kernel(const float *__restrict__ x, uint64_t n, double *out) {
    const int c = blockIdx.x;
    double s = 0, q = 0;
    for (uint64_t r = threadIdx.x; r < n; r += blockDim.x) {
        const double v = x[r * IN + c];
        s += v;
        q += v * v;
    }
    __shared__ double rs[256], rq[256];
    rs[threadIdx.x] = s;
    rq[threadIdx.x] = q;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            rs[threadIdx.x] += rs[threadIdx.x + o];
            rq[threadIdx.x] += rq[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[2 * c] = rs[0];
        out[2 * c + 1] = rq[0];
    }
}

}  // namespace arso

struct arso_surrogate {
    arso::DeviceBuffer w, w16, m, v, g, norm;
    float mean[arso::IN], sd[arso::IN];
    bool norm_set = false;
    uint64_t t = 0;
};

namespace arso {

struct Activations {
    DeviceBuffer xb, h1, h2, z, dz, dh1, dh2, lsum;
    int cap = 0;
    void ensure(int rows) {
        if (rows <= cap) return;
        xb.ensure((size_t)rows * IN * 4);
        h1.ensure((size_t)rows * HID * 4);
        h2.ensure((size_t)rows * HID * 4);
        z.ensure((size_t)rows * 4);
        dz.ensure((size_t)rows * 4);
        dh1.ensure((size_t)rows * HID * 4);
        dh2.ensure((size_t)rows * HID * 4);
        lsum.ensure(8);
        cap = rows;
    }
};

static void upload_norm(arso_surrogate *s) {
    float h[2 * IN];
    std::memcpy(h, s->mean, sizeof(s->mean));
    std::memcpy(h + IN, s->sd, sizeof(s->sd));
    s->norm.ensure(sizeof(h));
    ARSO_CUDA(cudaMemcpy(s->norm.ptr, h, sizeof(h), cudaMemcpyHostToDevice));
}

// forward of `rows` gathered rows: xb -> h1 -> h2 -> z (logits)
static void mlp_forward(const arso_surrogate *s, Activations &a, int rows, cudaStream_t st) {
    const __nv_bfloat16 *w = s->w16.as<__nv_bfloat16>();
    gemm<float, __nv_bfloat16>(rows, HID, IN, a.xb.as<float>(), IN, 1, w + OFF_W1, HID, 1, a.h1.as<float>(),
                               EPI_BIAS_RELU, w + OFF_B1, nullptr, st);
    gemm<float, __nv_bfloat16>(rows, HID, HID, a.h1.as<float>(), HID, 1, w + OFF_W2, HID, 1, a.h2.as<float>(),
                               EPI_BIAS_RELU, w + OFF_B2, nullptr, st);
    gemm<float, __nv_bfloat16>(rows, 1, HID, a.h2.as<float>(), HID, 1, w + OFF_W3, 1, 1, a.z.as<float>(), EPI_BIAS,
                               w + OFF_B3, nullptr, st);
}

// gradients of the mean BCE into s->g (FP32) given a.dz
static void mlp_backward(const arso_surrogate *s, Activations &a, int rows, float *g, cudaStream_t st) {
    const __nv_bfloat16 *w = s->w16.as<__nv_bfloat16>();
    // dW3[k] = sum_i h2[i,k] dz[i]; db3 = sum_i dz[i]
    gemm<float, float>(HID, 1, rows, a.h2.as<float>(), 1, HID, a.dz.as<float>(), 1, 1, g + OFF_W3, EPI_NONE, nullptr,
                       nullptr, st);
    colsum_kernel<<<1, 32, 0, st>>>(a.dz.as<float>(), rows, 1, g + OFF_B3);
    // dh2[i,k] = dz[i] W3[k] (h2 > 0)
    gemm<float, __nv_bfloat16>(rows, HID, 1, a.dz.as<float>(), 1, 1, w + OFF_W3, 1, 1, a.dh2.as<float>(),
                               EPI_RELU_MASK, nullptr, a.h2.as<float>(), st);
    // dW2 = h1^T dh2; db2 = colsum dh2
    gemm<float, float>(HID, HID, rows, a.h1.as<float>(), 1, HID, a.dh2.as<float>(), HID, 1, g + OFF_W2, EPI_NONE,
                       nullptr, nullptr, st);
    colsum_kernel<<<(HID + 127) / 128, 128, 0, st>>>(a.dh2.as<float>(), rows, HID, g + OFF_B2);
    // dh1 = dh2 W2^T (h1 > 0)
    gemm<float, __nv_bfloat16>(rows, HID, HID, a.dh2.as<float>(), HID, 1, w + OFF_W2, 1, HID, a.dh1.as<float>(),
                               EPI_RELU_MASK, nullptr, a.h1.as<float>(), st);
    // dW1 = xb^T dh1; db1 = colsum dh1
    gemm<float, float>(IN, HID, rows, a.xb.as<float>(), 1, IN, a.dh1.as<float>(), HID, 1, g + OFF_W1, EPI_NONE,
                       nullptr, nullptr, st);
    colsum_kernel<<<(HID + 127) / 128, 128, 0, st>>>(a.dh1.as<float>(), rows, HID, g + OFF_B1);
    ARSO_CUDA(cudaGetLastError());
}

static void refresh_bf16(arso_surrogate *s, cudaStream_t st) {
    to_bf16_kernel<<<64, 256, 0, st>>>(s->w.as<float>(), s->w16.as<__nv_bfloat16>(), N_PARAMS);
    ARSO_CUDA(cudaGetLastError());
}

static void ensure_norm(arso_surrogate *s, const float *x, uint64_t n, cudaStream_t st) {
    if (s->norm_set) return;
    DeviceBuffer mom;
    mom.ensure(2 * IN * sizeof(double));
    moments_kernel<<<IN, 256, 0, st>>>(x, n, mom.as<double>());
    ARSO_CUDA(cudaGetLastError());
    double h[2 * IN];
    ARSO_CUDA(cudaMemcpyAsync(h, mom.ptr, sizeof(h), cudaMemcpyDeviceToHost, st));
    ARSO_CUDA(cudaStreamSynchronize(st));
    for (int c = 0; c < IN; ++c) {
        const double mu = h[2 * c] / (double)n;
        const double var = std::max(0.0, h[2 * c + 1] / (double)n - mu * mu);
        s->mean[c] = (float)mu;
        s->sd[c] = var > 1e-12 ? (float)std::sqrt(var) : 1.f;
    }
    s->norm_set = true;
    upload_norm(s);
}

}  // namespace arso

using namespace arso;

extern "C" {

arso_status arso_surrogate_create(uint64_t seed, arso_surrogate **out) {
    try {
        ARSO_REQUIRE(out != nullptr, "out is NULL");
        std::unique_ptr<arso_surrogate> s(new arso_surrogate());
        std::vector<float> h(N_PARAMS, 0.f);
        std::mt19937_64 rng(seed);
        auto fill = [&](size_t off, int fan_in, size_t cnt) {
            const double lim = std::sqrt(6.0 / fan_in);  // He-uniform
            std::uniform_real_distribution<double> U(-lim, lim);
            for (size_t i = 0; i < cnt; ++i) h[off + i] = (float)U(rng);
        };
        fill(OFF_W1, IN, (size_t)IN * HID);
        fill(OFF_W2, HID, (size_t)HID * HID);
        fill(OFF_W3, HID, HID);
        s->w.ensure(N_PARAMS * 4);
        s->w16.ensure(N_PARAMS * 2);
        s->m.ensure(N_PARAMS * 4);
        s->v.ensure(N_PARAMS * 4);
        s->g.ensure(N_PARAMS * 4);
        ARSO_CUDA(cudaMemcpy(s->w.ptr, h.data(), N_PARAMS * 4, cudaMemcpyHostToDevice));
        ARSO_CUDA(cudaMemset(s->m.ptr, 0, N_PARAMS * 4));
        ARSO_CUDA(cudaMemset(s->v.ptr, 0, N_PARAMS * 4));
        for (int c = 0; c < IN; ++c) s->mean[c] = 0.f, s->sd[c] = 1.f;
        upload_norm(s.get());
        refresh_bf16(s.get(), 0);
        ARSO_CUDA(cudaDeviceSynchronize());
        *out = s.release();
        return ARSO_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    }
}

void arso_surrogate_free(arso_surrogate *s) { delete s; }

arso_status arso_surrogate_set_norm(arso_surrogate *s, const float *mean, const float *stdev) {
    try {
        ARSO_REQUIRE(s && mean && stdev, "NULL argument");
        for (int c = 0; c < IN; ++c) {
            ARSO_REQUIRE(stdev[c] > 0.f, "standard deviations must be positive");
            s->mean[c] = mean[c];
            s->sd[c] = stdev[c];
        }
        s->norm_set = true;
        upload_norm(s);
        return ARSO_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    }
}

arso_status arso_surrogate_get_params(const arso_surrogate *s, float *out) {
    try {
        ARSO_REQUIRE(s && out, "NULL argument");
        ARSO_CUDA(cudaMemcpy(out, s->w.ptr, N_PARAMS * 4, cudaMemcpyDeviceToHost));
        return ARSO_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    }
}

arso_status arso_surrogate_set_params(arso_surrogate *s, const float *in) {
    try {
        ARSO_REQUIRE(s && in, "NULL argument");
        ARSO_CUDA(cudaMemcpy(s->w.ptr, in, N_PARAMS * 4, cudaMemcpyHostToDevice));
        refresh_bf16(s, 0);
        ARSO_CUDA(cudaDeviceSynchronize());
        return ARSO_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    }
}

arso_status arso_surrogate_grads(const arso_surrogate *s, const float *x, const float *y, uint64_t n, void *stream,
                                 float *grads_out, double *loss_out) {
    try {
        ARSO_REQUIRE(s && x && y && grads_out, "NULL argument");
        ARSO_REQUIRE(n > 0 && n <= (1u << 20), "n must be in [1, 2^20]");
        cudaStream_t st = (cudaStream_t)stream;
        Activations a;
        a.ensure((int)n);
        ProfScope ps_(ARSO_K_OTHER, 0.0, st);
        gather_norm_kernel<<<(unsigned)n, 64, 0, st>>>(x, nullptr, 0, (int)n, s->norm.as<float>(), a.xb.as<float>());
        mlp_forward(s, a, (int)n, st);
        ARSO_CUDA(cudaMemsetAsync(a.lsum.ptr, 0, 8, st));
        bce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a.z.as<float>(), y, nullptr, 0, (int)n, 1.f / (float)n,
                                                                a.dz.as<float>(), a.lsum.as<double>());
        DeviceBuffer g;
        g.ensure(N_PARAMS * 4);
        mlp_backward(s, a, (int)n, g.as<float>(), st);
        ARSO_CUDA(cudaMemcpyAsync(grads_out, g.ptr, N_PARAMS * 4, cudaMemcpyDeviceToHost, st));
        double l = 0;
        ARSO_CUDA(cudaMemcpyAsync(&l, a.lsum.ptr, 8, cudaMemcpyDeviceToHost, st));
        ARSO_CUDA(cudaStreamSynchronize(st));
        if (loss_out) *loss_out = l / (double)n;
        return ARSO_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    }
}

arso_status arso_surrogate_train(arso_surrogate *s, const float *x, const float *y, uint64_t n, uint32_t epochs,
                                 uint32_t batch, double lr, uint64_t seed, void *stream, double *loss_out) {
    try {
        ARSO_REQUIRE(s && x && y, "NULL argument");
        ARSO_REQUIRE(n > 0 && n < (1ull << 32), "n must be in [1, 2^32)");
        ARSO_REQUIRE(batch > 0 && batch <= 65536, "batch must be in [1, 65536]");
        ARSO_REQUIRE(lr > 0, "lr must be > 0");
        cudaStream_t st = (cudaStream_t)stream;
        ensure_norm(s, x, n, st);
        Activations a;
        a.ensure((int)std::min<uint64_t>(batch, n));
        DeviceBuffer d_idx;
        d_idx.ensure(n * 4);
        std::vector<uint32_t> idx(n);
        std::mt19937_64 rng(seed);
        double last = 0;
        for (uint32_t ep = 0; ep < epochs; ++ep) {
            for (uint64_t i = 0; i < n; ++i) idx[i] = (uint32_t)i;
            std::shuffle(idx.begin(), idx.end(), rng);
            ARSO_CUDA(cudaMemcpyAsync(d_idx.ptr, idx.data(), n * 4, cudaMemcpyHostToDevice, st));
            ARSO_CUDA(cudaMemsetAsync(a.lsum.ptr, 0, 8, st));
            for (uint64_t b0 = 0; b0 < n; b0 += batch) {
                const int rows = (int)std::min<uint64_t>(batch, n - b0);
                ProfScope ps_(ARSO_K_OTHER, 0.0, st);
                gather_norm_kernel<<<rows, 64, 0, st>>>(x, d_idx.as<uint32_t>(), b0, rows, s->norm.as<float>(),
                                                        a.xb.as<float>());
                mlp_forward(s, a, rows, st);
                bce_kernel<<<(rows + 255) / 256, 256, 0, st>>>(a.z.as<float>(), y, d_idx.as<uint32_t>(), b0, rows,
                                                              1.f / (float)rows, a.dz.as<float>(), a.lsum.as<double>());
                mlp_backward(s, a, rows, s->g.as<float>(), st);
                s->t += 1;
                const float c1 = 1.f - (float)std::pow(0.9, (double)s->t), c2 = 1.f - (float)std::pow(0.999, (double)s->t);
                adam_kernel<<<152, 256, 0, st>>>(s->w.as<float>(), s->w16.as<__nv_bfloat16>(), s->g.as<float>(),
                                                 s->m.as<float>(), s->v.as<float>(), N_PARAMS, (float)lr, 0.9f, 0.999f,
                                                 1e-8f, c1, c2);
                ARSO_CUDA(cudaGetLastError());
            }
            ARSO_CUDA(cudaMemcpyAsync(&last, a.lsum.ptr, 8, cudaMemcpyDeviceToHost, st));
            ARSO_CUDA(cudaStreamSynchronize(st));
        }
        if (loss_out) *loss_out = last / (double)n;
        return ARSO_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    }
}

arso_status arso_surrogate_predict(const arso_surrogate *s, const float *x, uint64_t n, float *out, void *stream) {
    try {
        ARSO_REQUIRE(s && x && out, "NULL argument");
        cudaStream_t st = (cudaStream_t)stream;
        Activations a;
        const uint64_t chunk = 65536;
        a.ensure((int)std::min<uint64_t>(n, chunk));
        for (uint64_t b0 = 0; b0 < n; b0 += chunk) {
            const int rows = (int)std::min<uint64_t>(chunk, n - b0);
            ProfScope ps_(ARSO_K_OTHER, 0.0, st);
            gather_norm_kernel<<<rows, 64, 0, st>>>(x, nullptr, b0, rows, s->norm.as<float>(), a.xb.as<float>());
            mlp_forward(s, a, rows, st);
            sigmoid_kernel<<<(rows + 255) / 256, 256, 0, st>>>(a.z.as<float>(), rows, out + b0);
            ARSO_CUDA(cudaGetLastError());
        }
        ARSO_CUDA(cudaStreamSynchronize(st));
        return ARSO_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    }
}

arso_status arso_circuit_features(const arso_circuit *c, const arso_criterion *crit, float *out) {
    try {
        ARSO_REQUIRE(c && crit && out, "NULL argument");
        const std::vector<float> f = circuit_features(c, crit);
        std::copy(f.begin(), f.end(), out);
        return ARSO_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    }
}

}  // extern "C"
