// model.cu -- the entry-context model of the speculative path: a byte-window
// network that reads the 64 bytes around a chunk start and scores every
// context (BOUNDARY or a DFA state), trained on the true contexts that the
// enumerative path resolves.  The lexer stays exact whatever it predicts: a
// wrong guess only costs a rescan.
//
//   h0[t]   = emb[x_t]                               x = w[p - 32, p + 32), pad byte 256 outside
//   a[t,f]  = bc[f] + sum_{k<5,d<8} Wc[f,k,d] h0[t+k-2,d]   (zero outside the window)
//   m[u,f]  = max_{t=4u..4u+3} relu(a[t,f])          (the first maximum takes the gradient)
//   h1      = relu(m W1 + b1),  z = h1 W2 + b2       W1: 512 x H, W2: H x C (C = states + 1)
//   loss    = mean over the batch of -log softmax(z)[y]
// 32 filters, H = 64 and the 211 contexts of the refused C-like set give
// 49 915 parameters.  Every product reads BF16 weights and accumulates in
// FP32 (activations stay FP32); FP32 master weights are updated by AdamW
// (decoupled weight decay on the weight matrices).  Inference takes the
// argmax of z over the candidate contexts of the byte before p.  The products
// are small (a few hundred MFLOP per 512 MiB of input) and run on the CUDA
// cores.

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"
#include "runtime.h"

namespace lx {
namespace {

constexpr uint32_t MW = 64;          // window bytes
constexpr uint32_t MD = 8;           // embedding width
constexpr uint32_t MROWS = 257;      // 256 byte values + padding
constexpr uint32_t MF = 32;          // convolution filters
constexpr uint32_t MK = 5;           // filter width
constexpr uint32_t MPOOL = 4;        // max-pool width (and stride)
constexpr uint32_t MU = MW / MPOOL;  // pooled positions
constexpr uint32_t MIN_ = MU * MF;   // MLP input width (512)
constexpr int GT = 16;               // GEMM tile
constexpr uint32_t PRED_BATCH = 16384;
constexpr float WEIGHT_DECAY = 1e-2f;   // AdamW, on Wc, W1 and W2

}  // namespace
}  // namespace lx

struct lx_model {
    uint32_t C = 0, H = 0;
    uint64_t step = 0;
    // parameters in one FP32 block: emb | Wc | bc | W1 | b1 | W2 | b2, and Adam moments
    float *w = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;
    __nv_bfloat16 *w16 = nullptr;   // the BF16 weights every product reads
    size_t n_params = 0;
    size_t o_emb = 0, o_wc = 0, o_bc = 0, o_w1 = 0, o_b1 = 0, o_w2 = 0, o_b2 = 0;
    uint8_t *arg = nullptr;         // per (window, pooled position, filter): argmax | relu-active << 2
    size_t arg_bytes = 0;
    // activations for a batch, and windows for inference batches
    float *act = nullptr;
    size_t act_floats = 0;
    uint16_t *win = nullptr;
    int device = -1;
};

namespace lx {
namespace {

__device__ __forceinline__ uint32_t window_byte(const uint8_t *in, uint64_t n, uint64_t p, uint32_t k)
{
    const int64_t q = (int64_t)p - (int64_t)(MW / 2) + (int64_t)k;
    return (q >= 0 && (uint64_t)q < n) ? (uint32_t)in[q] : 256u;
}

__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }

// Convolution, ReLU and max pooling, one thread per (window, pooled
// position u, filter f): the four convolution outputs t = 4u .. 4u+3 over
// the eight embedded bytes they touch, the first maximum of their ReLU into
// m[b, u * MF + f], and its index (with whether it was positive) for the
// backward pass.
template <class TW>
__global__ void k_conv_pool(const uint16_t *win, uint32_t B, const TW *emb, const TW *wc, const TW *bc, float *mo,
                            uint8_t *arg)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * MIN_) return;
    const uint32_t b = i / MIN_, r = i % MIN_, u = r / MF, f = r % MF;
    float h[MPOOL + MK - 1][MD];
#pragma unroll
    for (uint32_t j = 0; j < MPOOL + MK - 1; j++) {
        const int t = (int)(u * MPOOL + j) - (int)(MK / 2);
        const bool in = t >= 0 && t < (int)MW;
        const uint32_t x = in ? win[(size_t)b * MW + t] : 0u;
#pragma unroll
        for (uint32_t d = 0; d < MD; d++) h[j][d] = in ? to_f(emb[(size_t)x * MD + d]) : 0.0f;
    }
    float best = -1.0f;
    uint32_t bj = 0, pos = 0;
#pragma unroll
    for (uint32_t j = 0; j < MPOOL; j++) {
        float a = to_f(bc[f]);
#pragma unroll
        for (uint32_t k = 0; k < MK; k++)
#pragma unroll
            for (uint32_t d = 0; d < MD; d++) a = fmaf(to_f(wc[((size_t)f * MK + k) * MD + d]), h[j + k][d], a);
        const float rr = a > 0.0f ? a : 0.0f;
        if (rr > best) {
            best = rr;
            bj = j;
            pos = a > 0.0f ? 1u : 0u;
        }
    }
    mo[i] = best;
    if (arg) arg[i] = (uint8_t)(bj | (pos << 2));
}

// Backward through pooling and the convolution's weights: each thread one
// (f, k, d) weight over a slice of the batch (and thread d == 0, k == 0 the
// bias), atomically accumulated.  dm: gradient of m.
template <class TW>
__global__ void k_conv_back_w(const uint16_t *win, uint32_t B, const TW *emb, const float *dm, const uint8_t *arg,
                              float *gwc, float *gbc, uint32_t per)
{
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= MF * MK * MD) return;
    const uint32_t f = q / (MK * MD), k = (q / MD) % MK, d = q % MD;
    const uint32_t b0 = blockIdx.y * per, b1 = min(B, b0 + per);
    float sw = 0.0f, sb = 0.0f;
    for (uint32_t b = b0; b < b1; b++)
        for (uint32_t u = 0; u < MU; u++) {
            const uint32_t i = b * MIN_ + u * MF + f;
            const uint32_t ar = arg[i];
            if (!(ar & 4u)) continue;
            const float da = dm[i];
            sb += da;
            const int t = (int)(u * MPOOL + (ar & 3u) + k) - (int)(MK / 2);
            if (t >= 0 && t < (int)MW) sw = fmaf(da, to_f(emb[(size_t)win[(size_t)b * MW + t] * MD + d]), sw);
        }
    atomicAdd(&gwc[q], sw);
    if (k == 0 && d == 0) atomicAdd(&gbc[f], sb);
}

// Backward through the convolution's input: dh0[b, t, d] from every pooled
// maximum whose filter touched t; one thread per (window, u, f).
template <class TW>
__global__ void k_conv_back_x(uint32_t B, const TW *wc, const float *dm, const uint8_t *arg, float *dh0)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * MIN_) return;
    const uint32_t ar = arg[i];
    if (!(ar & 4u)) return;
    const uint32_t b = i / MIN_, r = i % MIN_, u = r / MF, f = r % MF;
    const float da = dm[i];
    for (uint32_t k = 0; k < MK; k++) {
        const int t = (int)(u * MPOOL + (ar & 3u) + k) - (int)(MK / 2);
        if (t < 0 || t >= (int)MW) continue;
        for (uint32_t d = 0; d < MD; d++)
            atomicAdd(&dh0[((size_t)b * MW + t) * MD + d], da * to_f(wc[((size_t)f * MK + k) * MD + d]));
    }
}

// C[M x N] = alpha * op(A) op(B) (+ bias[N]) (+ C if accumulate): A is M x K
// (or K x M when ta), B is K x N (or N x K when tb), all row-major.
template <class TW>
__global__ void k_gemm(const float *A, const TW *Bm, float *Cm, const TW *bias, uint32_t M, uint32_t N,
                       uint32_t K, int ta, int tb, int relu_out)
{
    __shared__ float As[GT][GT + 1], Bs[GT][GT + 1];
    const uint32_t r = blockIdx.y * GT + threadIdx.y, c = blockIdx.x * GT + threadIdx.x;
    float acc = 0.0f;
    for (uint32_t k0 = 0; k0 < K; k0 += GT) {
        const uint32_t ka = k0 + threadIdx.x, kb = k0 + threadIdx.y;
        As[threadIdx.y][threadIdx.x] =
            (r < M && ka < K) ? (ta ? A[(size_t)ka * M + r] : A[(size_t)r * K + ka]) : 0.0f;
        Bs[threadIdx.y][threadIdx.x] =
            (kb < K && c < N) ? to_f(tb ? Bm[(size_t)c * K + kb] : Bm[(size_t)kb * N + c]) : 0.0f;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < GT; k++) acc = fmaf(As[threadIdx.y][k], Bs[k][threadIdx.x], acc);
        __syncthreads();
    }
    if (r < M && c < N) {
        if (bias) acc += to_f(bias[c]);
        if (relu_out) acc = acc > 0.0f ? acc : 0.0f;
        Cm[(size_t)r * N + c] = acc;
    }
}

// Inference products: C[M x N] = A[M x K] B[K x N] + bias (ReLU optional),
// each CTA a 64 x 64 tile of C, each thread a 4 x 4 block of it in
// registers, K in steps of 16 through shared memory.
constexpr int RB_T = 64, RB_K = 16;

template <class TW>
__global__ void __launch_bounds__(256) k_gemm_rb(const float *A, const TW *Bm, float *Cm, const TW *bias, uint32_t M,
                                                 uint32_t N, uint32_t K, int relu_out)
{
    __shared__ __align__(16) float As[RB_K][RB_T + 4];   // A tile, k-major
    __shared__ __align__(16) float Bs[RB_K][RB_T + 4];
    const uint32_t tid = threadIdx.x, tx = tid & 15u, ty = tid >> 4;
    const uint32_t m0 = blockIdx.y * RB_T, n0 = blockIdx.x * RB_T;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = 0.0f;
    for (uint32_t k0 = 0; k0 < K; k0 += RB_K) {
        {
            const uint32_t r = tid >> 2, kk = (tid & 3u) * 4u, m = m0 + r;
#pragma unroll
            for (uint32_t i = 0; i < 4; i++) {
                const uint32_t k = k0 + kk + i;
                float v = 0.0f;
                if (m < M && k < K) v = A[(size_t)m * K + k];
                As[kk + i][r] = v;
            }
        }
        {
            const uint32_t kr = tid >> 4, c = (tid & 15u) * 4u, k = k0 + kr;
#pragma unroll
            for (uint32_t i = 0; i < 4; i++) {
                const uint32_t nn = n0 + c + i;
                Bs[kr][c + i] = (k < K && nn < N) ? to_f(Bm[(size_t)k * N + nn]) : 0.0f;
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < RB_K; k++) {
            const float4 a = *reinterpret_cast<const float4 *>(&As[k][ty * 4]);
            const float4 b = *reinterpret_cast<const float4 *>(&Bs[k][tx * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const uint32_t m = m0 + ty * 4 + i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const uint32_t nn = n0 + tx * 4 + j;
            if (nn >= N) continue;
            float v = acc[i][j];
            if (bias) v += to_f(bias[nn]);
            if (relu_out) v = v > 0.0f ? v : 0.0f;
            Cm[(size_t)m * N + nn] = v;
        }
    }
}

// softmax cross-entropy per row: dz = (softmax(z) - onehot(y)) / B, loss sum
__global__ void k_softmax_ce(const float *z, const uint16_t *y, uint32_t B, uint32_t C, float *dz, float *loss)
{
    const uint32_t b = blockIdx.x;
    if (b >= B) return;
    const float *zr = z + (size_t)b * C;
    float mx = -INFINITY;
    for (uint32_t c = threadIdx.x; c < C; c += blockDim.x) mx = fmaxf(mx, zr[c]);
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    float se = 0.0f;
    for (uint32_t c = threadIdx.x; c < C; c += blockDim.x) se += expf(zr[c] - mx);
    for (int o = 16; o; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
    const float lse = mx + logf(se);
    for (uint32_t c = threadIdx.x; c < C; c += blockDim.x) {
        const float pr = expf(zr[c] - lse);
        dz[(size_t)b * C + c] = (pr - (c == y[b] ? 1.0f : 0.0f)) / (float)B;
    }
    if (threadIdx.x == 0) atomicAdd(loss, (lse - zr[y[b]]) / (float)B);
}

// column sums: out[c] = sum_b M[b, c]
__global__ void k_colsum(const float *Mx, uint32_t B, uint32_t N, float *out)
{
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    float s = 0.0f;
    for (uint32_t b = 0; b < B; b++) s += Mx[(size_t)b * N + c];
    out[c] = s;
}

// dA1 = dH1 * (A1 > 0)
__global__ void k_relu_back(float *dh, const float *a, size_t n)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && a[i] <= 0.0f) dh[i] = 0.0f;
}

// demb[x, d] += dh0[b, t, d] for byte x at window position t
__global__ void k_emb_back(const uint16_t *win, uint32_t B, const float *dh0, float *demb)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * MW * MD) return;
    const uint32_t b = i / (MW * MD), r = i % (MW * MD), t = r / MD, d = r % MD;
    const float v = dh0[i];
    if (v != 0.0f) atomicAdd(&demb[(size_t)win[(size_t)b * MW + t] * MD + d], v);
}

// AdamW (beta 0.9 / 0.999, eps 1e-8): decoupled weight decay on the weight
// matrices [d0, d1), [d2, d3), [d4, d5), then the Adam step; the BF16 copy
// follows the FP32 master weights.
__global__ void k_adamw(float *w, float *m, float *v, const float *g, __nv_bfloat16 *w16, size_t n, float lr,
                        float b1c, float b2c, float wd, size_t d0, size_t d1, size_t d2, size_t d3, size_t d4,
                        size_t d5)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    float wi = w[i];
    if ((i >= d0 && i < d1) || (i >= d2 && i < d3) || (i >= d4 && i < d5)) wi -= lr * wd * wi;
    wi -= lr * (mi / b1c) / (sqrtf(vi / b2c) + 1e-8f);
    w[i] = wi;
    w16[i] = __float2bfloat16(wi);
}

__global__ void k_to_bf16(const float *w, __nv_bfloat16 *w16, size_t n)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) w16[i] = __float2bfloat16(w[i]);
}

// windows of the chunk starts (pad where there is no start)
__global__ void k_windows(const uint8_t *in, uint64_t n, const uint64_t *start, uint32_t j0, uint32_t cnt,
                          uint16_t *win)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt * MW) return;
    const uint32_t b = i / MW, k = i % MW;
    const uint64_t p = start[j0 + b];
    win[i] = p == ~0ull ? 256u : (uint16_t)window_byte(in, n, p, k);
}

// The argmax of the logits over the candidate contexts of the byte before
// each chunk start (BOUNDARY = class C-1 -> 0xFFFE); one warp per chunk.
__global__ void k_argmax(const float *z, uint32_t C, uint32_t j0, uint32_t cnt, const uint64_t *start,
                         const uint32_t *cinfo, const uint8_t *scan_blob, uint32_t cbeg_off, uint32_t cand_off,
                         uint16_t *guess)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (b >= cnt) return;
    const uint32_t j = j0 + b;
    if (j == 0 || start[j] == ~0ull) {
        if (lane == 0) guess[j] = 0xFFFEu;
        return;
    }
    const uint16_t *cbeg = reinterpret_cast<const uint16_t *>(scan_blob + cbeg_off);
    const uint16_t *cand = reinterpret_cast<const uint16_t *>(scan_blob + cand_off);
    const uint32_t byte = cinfo[j] >> 8, lo = cbeg[byte], hi = cbeg[byte + 1];
    const float *zr = z + (size_t)b * C;
    float best = -INFINITY;
    uint32_t arg = C - 1;
    for (uint32_t t = lane; t < 1 + hi - lo; t += 32) {
        const uint32_t c = t == 0 ? C - 1 : cand[lo + t - 1];
        const float v = zr[c];
        if (v > best || (v == best && c < arg)) {
            best = v;
            arg = c;
        }
    }
    for (int o = 16; o; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const uint32_t oa = __shfl_xor_sync(0xffffffffu, arg, o);
        if (ob > best || (ob == best && oa < arg)) {
            best = ob;
            arg = oa;
        }
    }
    if (lane == 0) guess[j] = arg == C - 1 ? (uint16_t)0xFFFEu : (uint16_t)arg;
}

}  // namespace

uint32_t model_contexts(const lx_model *m) { return m ? m->C : 0; }

}  // namespace lx

using namespace lx;

namespace {

int ensure_act(lx_model *m, uint32_t B)
{
    const size_t need = (size_t)B * (MIN_ * 2 + MW * MD + m->H * 3 + m->C * 2) + 16;
    if (m->act_floats < need) {
        if (m->act) cudaFree(m->act);
        m->act = nullptr;
        m->act_floats = 0;
        if (cudaMalloc(&m->act, need * sizeof(float)) != cudaSuccess) return LX_E_NOMEM;
        m->act_floats = need;
    }
    const size_t abytes = (size_t)B * MIN_;
    if (m->arg_bytes < abytes) {
        if (m->arg) cudaFree(m->arg);
        m->arg = nullptr;
        m->arg_bytes = 0;
        if (cudaMalloc(&m->arg, abytes) != cudaSuccess) return LX_E_NOMEM;
        m->arg_bytes = abytes;
    }
    return LX_OK;
}

dim3 gemm_grid(uint32_t M, uint32_t N) { return dim3((N + GT - 1) / GT, (M + GT - 1) / GT); }
dim3 rb_grid(uint32_t M, uint32_t N) { return dim3((N + RB_T - 1) / RB_T, (M + RB_T - 1) / RB_T); }

// Forward (and with labels, backward into m->g) for a batch of windows, on
// the BF16 weights.  Activations: m | a1 | h1 | z | dz | dh1 | dm | dh0 | loss
int model_pass(lx_model *m, const uint16_t *d_win, const uint16_t *d_y, uint32_t B, float *d_logits_out,
               cudaStream_t s, float *h_loss)
{
    int rc = ensure_act(m, B);
    if (rc != LX_OK) return rc;
    const uint32_t H = m->H, C = m->C;
    float *mo = m->act, *a1 = mo + (size_t)B * MIN_, *h1 = a1 + (size_t)B * H, *z = h1 + (size_t)B * H;
    float *dz = z + (size_t)B * C, *dh1 = dz + (size_t)B * C, *dm = dh1 + (size_t)B * H;
    float *dh0 = dm + (size_t)B * MIN_, *loss = dh0 + (size_t)B * MW * MD;
    const __nv_bfloat16 *w = m->w16;
    const dim3 t2(GT, GT);
    const uint32_t nm = B * MIN_;
    k_conv_pool<__nv_bfloat16><<<(nm + 255) / 256, 256, 0, s>>>(d_win, B, w + m->o_emb, w + m->o_wc, w + m->o_bc, mo,
                                                               m->arg);
    k_gemm<__nv_bfloat16><<<gemm_grid(B, H), t2, 0, s>>>(mo, w + m->o_w1, a1, w + m->o_b1, B, H, MIN_, 0, 0, 0);
    cudaMemcpyAsync(h1, a1, sizeof(float) * B * H, cudaMemcpyDeviceToDevice, s);
    k_relu_back<<<(B * H + 255) / 256, 256, 0, s>>>(h1, a1, (size_t)B * H);   // h1 = relu(a1)
    k_gemm<__nv_bfloat16><<<gemm_grid(B, C), t2, 0, s>>>(h1, w + m->o_w2, z, w + m->o_b2, B, C, H, 0, 0, 0);
    if (d_logits_out)
        cudaMemcpyAsync(d_logits_out, z, sizeof(float) * B * C, cudaMemcpyDeviceToDevice, s);
    if (!d_y) return cuda_err(cudaGetLastError());
    float *g = m->g;
    cudaMemsetAsync(loss, 0, sizeof(float), s);
    cudaMemsetAsync(g, 0, sizeof(float) * m->n_params, s);
    cudaMemsetAsync(dh0, 0, sizeof(float) * B * MW * MD, s);
    k_softmax_ce<<<B, 32, 0, s>>>(z, d_y, B, C, dz, loss);
    k_gemm<float><<<gemm_grid(H, C), t2, 0, s>>>(h1, dz, g + m->o_w2, nullptr, H, C, B, 1, 0, 0);   // h1^T dz
    k_colsum<<<(C + 255) / 256, 256, 0, s>>>(dz, B, C, g + m->o_b2);
    k_gemm<__nv_bfloat16><<<gemm_grid(B, H), t2, 0, s>>>(dz, w + m->o_w2, dh1, nullptr, B, H, C, 0, 1, 0);  // dz W2^T
    k_relu_back<<<(B * H + 255) / 256, 256, 0, s>>>(dh1, a1, (size_t)B * H);
    k_gemm<float><<<gemm_grid(MIN_, H), t2, 0, s>>>(mo, dh1, g + m->o_w1, nullptr, MIN_, H, B, 1, 0, 0);  // m^T dh1
    k_colsum<<<(H + 255) / 256, 256, 0, s>>>(dh1, B, H, g + m->o_b1);
    k_gemm<__nv_bfloat16><<<gemm_grid(B, MIN_), t2, 0, s>>>(dh1, w + m->o_w1, dm, nullptr, B, MIN_, H, 0, 1, 0);
    const uint32_t per = 32;
    const dim3 gw((MF * MK * MD + 127) / 128, (B + per - 1) / per);
    k_conv_back_w<__nv_bfloat16><<<gw, 128, 0, s>>>(d_win, B, w + m->o_emb, dm, m->arg, g + m->o_wc, g + m->o_bc, per);
    k_conv_back_x<__nv_bfloat16><<<(nm + 255) / 256, 256, 0, s>>>(B, w + m->o_wc, dm, m->arg, dh0);
    k_emb_back<<<(B * MW * MD + 255) / 256, 256, 0, s>>>(d_win, B, dh0, g + m->o_emb);
    rc = cuda_err(cudaGetLastError());
    if (rc == LX_OK && h_loss) {
        rc = cuda_err(cudaMemcpyAsync(h_loss, loss, sizeof(float), cudaMemcpyDeviceToHost, s));
        if (rc == LX_OK) rc = cuda_err(cudaStreamSynchronize(s));
    }
    return rc;
}

// splitmix64 -> uniform in [-a, a)
float init_value(uint64_t &st, float a)
{
    st += 0x9E3779B97F4A7C15ull;
    uint64_t z = st;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (float)((double)(z >> 11) / (double)(1ull << 53) * 2.0 - 1.0) * a;
}

}  // namespace

int lx::model_predict(lx_model *m, const uint8_t *in, uint64_t n, const uint64_t *start, const uint32_t *cinfo,
                      const uint8_t *scan_blob, uint32_t cbeg_off, uint32_t cand_off, uint32_t M, uint16_t *guess,
                      cudaStream_t s)
{
    const uint32_t B = std::min<uint32_t>(M, PRED_BATCH);
    int rc = ensure_act(m, B);
    if (rc != LX_OK) return rc;
    if (!m->win && cudaMalloc(&m->win, sizeof(uint16_t) * PRED_BATCH * MW) != cudaSuccess) return LX_E_NOMEM;
    const uint32_t H = m->H, C = m->C;
    float *mo = m->act, *h1 = mo + (size_t)B * MIN_, *z = h1 + (size_t)B * H;
    const __nv_bfloat16 *w = m->w16;
    for (uint32_t j0 = 0; j0 < M; j0 += B) {
        const uint32_t cnt = std::min<uint32_t>(B, M - j0);
        k_windows<<<(cnt * MW + 255) / 256, 256, 0, s>>>(in, n, start, j0, cnt, m->win);
        k_conv_pool<__nv_bfloat16><<<(cnt * MIN_ + 255) / 256, 256, 0, s>>>(m->win, cnt, w + m->o_emb, w + m->o_wc,
                                                                           w + m->o_bc, mo, nullptr);
        // h1 = relu(m W1 + b1), z = h1 W2 + b2
        k_gemm_rb<__nv_bfloat16><<<rb_grid(cnt, H), 256, 0, s>>>(mo, w + m->o_w1, h1, w + m->o_b1, cnt, H, MIN_, 1);
        k_gemm_rb<__nv_bfloat16><<<rb_grid(cnt, C), 256, 0, s>>>(h1, w + m->o_w2, z, w + m->o_b2, cnt, C, H, 0);
        k_argmax<<<(cnt * 32 + 255) / 256, 256, 0, s>>>(z, C, j0, cnt, start, cinfo, scan_blob, cbeg_off, cand_off,
                                                        guess);
    }
    return cuda_err(cudaGetLastError());
}

extern "C" int lx_model_create(uint32_t n_contexts, uint32_t hidden, uint64_t seed, lx_model **out)
{
    if (!out || n_contexts < 2 || n_contexts > 0xFFFEu || hidden == 0 || hidden > 1024) return LX_E_INVAL;
    *out = nullptr;
    lx_model *m = new (std::nothrow) lx_model();
    if (!m) return LX_E_NOMEM;
    m->C = n_contexts;
    m->H = hidden;
    cudaGetDevice(&m->device);
    m->o_emb = 0;
    m->o_wc = m->o_emb + (size_t)MROWS * MD;
    m->o_bc = m->o_wc + (size_t)MF * MK * MD;
    m->o_w1 = m->o_bc + MF;
    m->o_b1 = m->o_w1 + (size_t)MIN_ * hidden;
    m->o_w2 = m->o_b1 + hidden;
    m->o_b2 = m->o_w2 + (size_t)hidden * n_contexts;
    m->n_params = m->o_b2 + n_contexts;
    std::vector<float> h(m->n_params, 0.0f);
    uint64_t st = seed;
    for (size_t i = m->o_emb; i < m->o_wc; i++) h[i] = init_value(st, 0.5f);
    const float ac = 1.0f / std::sqrt((float)(MK * MD)), a1 = 1.0f / std::sqrt((float)MIN_),
                a2 = 1.0f / std::sqrt((float)hidden);
    for (size_t i = m->o_wc; i < m->o_bc; i++) h[i] = init_value(st, ac);
    for (size_t i = m->o_w1; i < m->o_b1; i++) h[i] = init_value(st, a1);
    for (size_t i = m->o_w2; i < m->o_b2; i++) h[i] = init_value(st, a2);
    const size_t bytes = sizeof(float) * m->n_params;
    bool ok = cudaMalloc(&m->w, bytes) == cudaSuccess && cudaMalloc(&m->m, bytes) == cudaSuccess &&
              cudaMalloc(&m->v, bytes) == cudaSuccess && cudaMalloc(&m->g, bytes) == cudaSuccess &&
              cudaMalloc(&m->w16, sizeof(__nv_bfloat16) * m->n_params) == cudaSuccess;
    ok = ok && cudaMemcpy(m->w, h.data(), bytes, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(m->m, 0, bytes) == cudaSuccess && cudaMemset(m->v, 0, bytes) == cudaSuccess;
    if (ok) {
        k_to_bf16<<<(unsigned)((m->n_params + 255) / 256), 256>>>(m->w, m->w16, m->n_params);
        ok = cudaDeviceSynchronize() == cudaSuccess;
    }
    if (!ok) {
        lx_model_free(m);
        return LX_E_NOMEM;
    }
    *out = m;
    return LX_OK;
}

extern "C" void lx_model_free(lx_model *m)
{
    if (!m) return;
    cudaFree(m->w);
    cudaFree(m->m);
    cudaFree(m->v);
    cudaFree(m->g);
    cudaFree(m->w16);
    cudaFree(m->act);
    cudaFree(m->arg);
    cudaFree(m->win);
    delete m;
}

extern "C" int lx_model_info(const lx_model *m, uint32_t *n_contexts, uint32_t *hidden, uint32_t *window,
                             uint32_t *embed, uint64_t *n_params)
{
    if (!m) return LX_E_INVAL;
    if (n_contexts) *n_contexts = m->C;
    if (hidden) *hidden = m->H;
    if (window) *window = MW;
    if (embed) *embed = MD;
    if (n_params) *n_params = m->n_params;
    return LX_OK;
}

extern "C" int lx_model_get_params(const lx_model *m, float *host, uint64_t count)
{
    if (!m || !host || count != m->n_params) return LX_E_INVAL;
    return cuda_err(cudaMemcpy(host, m->w, sizeof(float) * count, cudaMemcpyDeviceToHost));
}

extern "C" int lx_model_set_params(lx_model *m, const float *host, uint64_t count)
{
    if (!m || !host || count != m->n_params) return LX_E_INVAL;
    int rc = cuda_err(cudaMemcpy(m->w, host, sizeof(float) * count, cudaMemcpyHostToDevice));
    if (rc != LX_OK) return rc;
    k_to_bf16<<<(unsigned)((m->n_params + 255) / 256), 256>>>(m->w, m->w16, m->n_params);
    return cuda_err(cudaDeviceSynchronize());
}

extern "C" int lx_model_windows(const uint8_t *d_in, uint64_t n, const uint64_t *d_pos, uint32_t count,
                                uint16_t *d_windows, void *stream)
{
    if ((count && (!d_pos || !d_windows)) || (n && !d_in)) return LX_E_INVAL;
    if (!count) return LX_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_windows<<<(count * MW + 255) / 256, 256, 0, s>>>(d_in, n, d_pos, 0, count, d_windows);
    return cuda_err(cudaGetLastError());
}

extern "C" int lx_model_forward(lx_model *m, const uint16_t *d_windows, uint32_t batch, float *d_logits,
                                void *stream)
{
    if (!m || !d_windows || !d_logits || batch == 0) return LX_E_INVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = model_pass(m, d_windows, nullptr, batch, d_logits, s, nullptr);
    if (rc == LX_OK) rc = cuda_err(cudaStreamSynchronize(s));
    return rc;
}

extern "C" int lx_model_gradient(lx_model *m, const uint16_t *d_windows, const uint16_t *d_labels, uint32_t batch,
                                 float *host_grad, uint64_t count, float *loss, void *stream)
{
    if (!m || !d_windows || !d_labels || batch == 0 || !host_grad || count != m->n_params) return LX_E_INVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float l = 0.0f;
    int rc = model_pass(m, d_windows, d_labels, batch, nullptr, s, &l);
    if (rc == LX_OK) rc = cuda_err(cudaMemcpy(host_grad, m->g, sizeof(float) * count, cudaMemcpyDeviceToHost));
    if (loss) *loss = l;
    return rc;
}

extern "C" int lx_model_train_step(lx_model *m, const uint16_t *d_windows, const uint16_t *d_labels,
                                   uint32_t batch, float lr, float *loss, void *stream)
{
    if (!m || !d_windows || !d_labels || batch == 0 || !(lr > 0.0f)) return LX_E_INVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float l = 0.0f;
    int rc = model_pass(m, d_windows, d_labels, batch, nullptr, s, &l);
    if (rc != LX_OK) return rc;
    m->step++;
    const float b1c = 1.0f - std::pow(0.9f, (float)m->step), b2c = 1.0f - std::pow(0.999f, (float)m->step);
    k_adamw<<<(unsigned)((m->n_params + 255) / 256), 256, 0, s>>>(m->w, m->m, m->v, m->g, m->w16, m->n_params, lr,
                                                                  b1c, b2c, WEIGHT_DECAY, m->o_wc, m->o_bc, m->o_w1,
                                                                  m->o_b1, m->o_w2, m->o_b2);
    rc = cuda_err(cudaGetLastError());
    if (loss) *loss = l;
    return rc;
}
