// Learned warm start of the pressure solve: a 4-level convolutional U-Net in
// BF16 on the tensor cores with FP32 accumulation, its training (forward,
// backward, Adam) and its use as the initial guess of a tank's solve.
//
// Every convolution is an implicit GEMM on tcgen05 with the accumulator in
// tensor memory: rows are output pixels, columns output channels, the reduction
// runs over (tap, input channel).  Activations and gradients are chunk-planar
// BF16 tensors ([rows][C / 8][W][8]).  The forward convolutions (3x3, nearest
// upsampling + 3x3, 2x2 stride 2) and the 3x3 input gradients (the 3x3
// convolution of the output gradient with the flipped, transposed weights) run
// in the halo kernels (k_conv_halo persistent and warp-specialised,
// k_conv_halo1 one tile per CTA): a stage holds one input row of one channel
// chunk, staged by bulk copy, and every horizontal tap reads it through a
// shifted descriptor; the weights of a stage arrive pre-packed in one bulk copy.
// The stride-2 layer's input gradient (one 1x1 GEMM per sub-pixel) gathers its
// operand with cp.async (k_conv_tc).  Weight gradients reduce over pixels, split
// across CTAs, with m16n8k16 MMAs (k_wgrad); their partial tiles are summed in a
// fixed order, so results are reproducible bit for bit.  ReLU masks, biases,
// the skip gradient and the BF16 rounding are fused into the GEMM epilogues.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "internal.cuh"
#include "poisson_op.cuh"
#include "tank.cuh"

typedef __nv_bfloat16 bf16;
typedef __nv_bfloat162 bf162;

namespace wec {
namespace {

// ------------------------------------------------------------ architecture --
enum LayerKind { L_CONV3 = 0, L_UP3 = 1, L_DOWN2 = 2, L_HEAD = 3 };

struct LayerDef {
    int kind, ci, co, level;  // level of the output tensor (0 = full resolution)
};

constexpr int kNumLayers = 21;
constexpr int kInCh = 2;   // features per cell
constexpr int kInPad = 16; // channels of the stored BF16 input (two 16-byte chunks per pixel)
const LayerDef kLayers[kNumLayers] = {
    {L_CONV3, 2, 32, 0},    {L_CONV3, 32, 32, 0},                           // enc0a, enc0b
    {L_DOWN2, 32, 64, 1},   {L_CONV3, 64, 64, 1},   {L_CONV3, 64, 64, 1},   // down0, enc1a, enc1b
    {L_DOWN2, 64, 128, 2},  {L_CONV3, 128, 128, 2}, {L_CONV3, 128, 128, 2}, // down1, enc2a, enc2b
    {L_DOWN2, 128, 256, 3}, {L_CONV3, 256, 256, 3}, {L_CONV3, 256, 256, 3}, // down2, enc3a, enc3b
    {L_UP3, 256, 128, 2},   {L_CONV3, 256, 128, 2}, {L_CONV3, 128, 128, 2}, // up2, cat2, dec2
    {L_UP3, 128, 64, 1},    {L_CONV3, 128, 64, 1},  {L_CONV3, 64, 64, 1},   // up1, cat1, dec1
    {L_UP3, 64, 32, 0},     {L_CONV3, 64, 32, 0},   {L_CONV3, 32, 32, 0},   // up0, cat0, dec0
    {L_HEAD, 32, 1, 0}};                                                    // head
constexpr int kHead = 20;
inline int enc_a(int l) { return 3 * l; }
inline int enc_b(int l) { return 3 * l + 1; }
inline int down(int l) { return 3 * l + 2; }      // l = 0..2: level l -> l + 1
inline int up(int l) { return 11 + 3 * (2 - l); }  // l = 2..0: level l + 1 -> l
inline int cat(int l) { return up(l) + 1; }
inline int dec(int l) { return up(l) + 2; }

inline int taps(int kind) { return kind == L_DOWN2 ? 4 : (kind == L_HEAD ? 1 : 9); }
inline int cin_pad(int ci) { return ci == kInCh ? kInPad : ci; }
inline int round_up(int a, int b) { return (a + b - 1) / b * b; }
inline size_t round_up_z(size_t a, size_t b) { return (a + b - 1) / b * b; }

// ----------------------------------------------------------- tile constants --
constexpr int kBM = 128;     // GEMM rows (pixels, or weight rows in k_wgrad) per CTA
constexpr int kBK = 32;      // reduction elements per pipeline stage
constexpr int kGT = 256;     // threads (8 warps: 4 along M x 2 along N)
constexpr int kStages = 3;

enum GatherKind { G_CONV3 = 0, G_UP3 = 1, G_DOWN2 = 2, G_DIRECT = 3 };
enum EpiKind { E_FWD = 0, E_DX = 1, E_F32 = 2, E_DOWNDX = 3 };

// A operand of a convolution as an implicit GEMM.  Row (n, i, j) of the N x H x
// W output grid, reduction index k = tap * cin + c with cin = c0 + c1 a power of
// two; channel c < c0 comes from in0, the rest from in1 (concatenation).
struct Gat {
    const bf16 *in0, *in1;
    int c0, c1, lcin;  // log2(cin)
    int kind;
    int N, H, W;       // output grid
    int Hi, Wi;        // grid of the input tensors
    int K;             // taps * cin; k >= K reads zeros (padding of the reduction)
};

// Fused epilogue.  E_FWD: out0 = bf16(relu(acc + bias)).  E_DX: input gradient;
// columns < nsplit: out0 = bf16(acc * (mask0 > 0)), the rest: out1 = bf16(acc).
// E_F32: outf = acc.  E_DOWNDX: the stride-2 layer's input gradient at the
// sub-pixel blockIdx.z of each row's 2x2 block: out0 = bf16((acc + add) * (mask0 > 0)).
struct Epi {
    int kind;
    const float *bias;
    bf16 *out0;
    const bf16 *mask0;
    int ld0;
    bf16 *out1;
    int ld1, nsplit;
    float *outf;
    const bf16 *add;
};

// ------------------------------------------------------------- PTX helpers --
__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

// 16-byte global -> shared copy; src_bytes = 0 fills the destination with zeros.
__device__ __forceinline__ void cp16(void *dst, const void *src, int src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ void ldm_x4_t(unsigned r[4], const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}

// d += a (16x16, row) * b (16x8, col), BF16 inputs, FP32 accumulators.
__device__ __forceinline__ void mma16816(float d[4], const unsigned a[4], const unsigned b[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// ---------------------------------------------------------- tensor layout --
// Activations and their gradients are chunk-planar BF16 tensors
// [rows][C / 8][W][8] (row = n H + y): the 8 channels [8q, 8q + 8) of a whole
// image row are contiguous, so a row segment of one channel chunk is one
// contiguous block (what the convolutions stage with bulk copies).
__device__ __forceinline__ size_t cofs(size_t row, int x, int c, int C, int W)
{
    return ((row * (size_t)(C >> 3) + (size_t)(c >> 3)) * (size_t)W + (size_t)x) * 8 + (size_t)(c & 7);
}

// ------------------------------------------------------------------ gather --
// Address of the 8 channels [c, c + 8) of reduction index k for output pixel
// (n, i, j), or nullptr where the operand is zero (outside the image, k >= K).
__device__ __forceinline__ const bf16 *gat_src(const Gat &g, int n, int i, int j, int k)
{
    if (k >= g.K) return nullptr;
    const int t = k >> g.lcin, c = k & ((1 << g.lcin) - 1);
    int ii = i, jj = j;
    if (g.kind == G_CONV3 || g.kind == G_UP3) {
        const int ta = t / 3, tb = t - 3 * ta;
        ii = i + ta - 1;
        jj = j + tb - 1;
        if (ii < 0 || jj < 0 || ii >= g.H || jj >= g.W) return nullptr;
        if (g.kind == G_UP3) {  // nearest upsampling: the input is the half grid
            ii >>= 1;
            jj >>= 1;
        }
    } else if (g.kind == G_DOWN2) {
        ii = 2 * i + (t >> 1);
        jj = 2 * j + (t & 1);
    }
    const size_t row = (size_t)n * g.Hi + ii;
    return c < g.c0 ? g.in0 + cofs(row, jj, c, g.c0, g.Wi) : g.in1 + cofs(row, jj, c - g.c0, g.c1, g.Wi);
}

__device__ __forceinline__ void epi_store(const Epi &e, const Gat &g, int p, int col, float v0, float v1)
{
    const size_t prow = (size_t)(p / g.W);
    const int px = p - (int)prow * g.W;
    if (e.kind == E_FWD) {
        v0 = fmaxf(v0 + e.bias[col], 0.0f);
        v1 = fmaxf(v1 + e.bias[col + 1], 0.0f);
        *reinterpret_cast<bf162 *>(e.out0 + cofs(prow, px, col, e.ld0, g.W)) = __floats2bfloat162_rn(v0, v1);
    } else if (e.kind == E_DX) {
        if (col < e.nsplit) {
            const size_t o = cofs(prow, px, col, e.ld0, g.W);
            const bf162 m = *reinterpret_cast<const bf162 *>(e.mask0 + o);
            v0 = __bfloat162float(m.x) > 0.0f ? v0 : 0.0f;
            v1 = __bfloat162float(m.y) > 0.0f ? v1 : 0.0f;
            *reinterpret_cast<bf162 *>(e.out0 + o) = __floats2bfloat162_rn(v0, v1);
        } else {
            *reinterpret_cast<bf162 *>(e.out1 + cofs(prow, px, col - e.nsplit, e.ld1, g.W)) =
                __floats2bfloat162_rn(v0, v1);
        }
    } else if (e.kind == E_F32) {
        *reinterpret_cast<float2 *>(e.outf + (size_t)p * e.ld0 + col) = make_float2(v0, v1);
    } else {  // E_DOWNDX: row p = (n, i, j) of the half grid -> (n, 2i + a, 2j + b)
        const int hw = g.H * g.W, n = p / hw, r = p - n * hw, i = r / g.W, j = r - i * g.W;
        const int a = blockIdx.z >> 1, b = blockIdx.z & 1;
        const size_t o = cofs((size_t)n * (2 * g.H) + 2 * i + a, 2 * j + b, col, e.ld0, 2 * g.W);
        const bf162 s = *reinterpret_cast<const bf162 *>(e.add + o);
        const bf162 m = *reinterpret_cast<const bf162 *>(e.mask0 + o);
        v0 = __bfloat162float(m.x) > 0.0f ? v0 + __bfloat162float(s.x) : 0.0f;
        v1 = __bfloat162float(m.y) > 0.0f ? v1 + __bfloat162float(s.y) : 0.0f;
        *reinterpret_cast<bf162 *>(e.out0 + o) = __floats2bfloat162_rn(v0, v1);
    }
}

// ------------------------------------------------- tcgen05 implicit GEMM --
// The same convolution GEMM on the 5th-generation tensor cores: one CTA owns a
// 128-pixel x BN-channel tile whose FP32 accumulator lives in tensor memory.
// Warps 0-3 gather A (one pixel row each) and B (K-major weights) into shared
// memory in the no-swizzle K-major core-matrix layout (8 rows x 16 bytes per
// core matrix; K-adjacent core matrices 128 B apart, 8-row groups 1024 B
// apart), kTcStages stages of 64 reduction elements; one thread of warp 4
// issues tcgen05.mma (M = 128, N = BN, K = 16, BF16 x BF16 -> FP32) and
// signals each consumed stage through tcgen05.commit.  Warps 0-3 then read
// their 32 TMEM lanes (tcgen05.ld) and run the fused epilogue.  Every wait is
// bounded: on expiry the kernel raises *err, drains its copies, frees its
// tensor memory and returns.
constexpr int kTcStages = 4;
constexpr int kTcK = 64;               // reduction elements per stage
constexpr int kTcThreads = 160;        // warps 0-3: producers / epilogue; warp 4: MMA
constexpr int kTcLag = 2;              // stages a producer keeps in flight before signalling
constexpr long long kWaitLimit = 1LL << 22;  // polls; far above any legitimate wait here

template <int BN>
struct TcSmem {
    static constexpr int kA = kBM * kTcK * 2;   // 16 KB
    static constexpr int kB = BN * kTcK * 2;
    static constexpr int kStage = kA + kB;
    static constexpr int kBytes = kTcStages * kStage + 256;  // + barriers and the TMEM address
};

__device__ __forceinline__ void mbar_init(unsigned a, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned a)
{
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(a) : "memory");
}
// Wait for the phase with the given parity to complete; false after kWaitLimit polls.
__device__ __forceinline__ bool mbar_wait(unsigned a, unsigned parity)
{
    for (long long it = 0; it < kWaitLimit; ++it) {
        unsigned ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ uint64_t umma_desc(unsigned saddr)
{
    // start address, K-direction core-matrix stride 128 B, 8-row-group stride
    // 1024 B (both >> 4), descriptor version 1 (bit 46), no swizzle
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           (1ull << 46);
}

template <int BN>
__host__ __device__ constexpr unsigned umma_idesc()
{
    // kind::f16: D F32 (bits 4-5 = 1), A BF16 (bits 7-9 = 1), B BF16 (bits 10-12 = 1),
    // both K-major, N >> 3 at bit 17, M >> 4 at bit 24
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(BN >> 3) << 17) | ((unsigned)(kBM >> 4) << 24);
}

// Epilogue of a tensor-core tile: the calling warp (warp = TMEM lane quarter)
// reads its 32 tile rows; tile row r is pixel m0 + r ps, valid below M.  The
// forward (bias + ReLU) and input-gradient (ReLU mask of the layer input, split
// into two outputs at nsplit) epilogues store each 8-channel chunk of a row as
// one 16-byte vector: the warp's 32 rows are consecutive pixels of one image
// row, so in the chunk-planar layout a warp's store of one chunk is contiguous.
// The others store pairs.  go is warp-uniform (tcgen05.ld is warp-collective).
template <int BN>
__device__ __forceinline__ void tc_epilogue(const Epi &e, const Gat &g, unsigned tmem, int m0, int n0, int M,
                                            int warp, int lane, bool go, int ps = 1)
{
    if (!go) return;
    const bool vec = e.kind == E_FWD || e.kind == E_DX;
    const int row = warp * 32 + lane, p = m0 + row * ps;
    const size_t prow = (size_t)(p / g.W);
    const int px = p - (int)prow * g.W;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
        unsigned v[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
            "[%16];\n"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c0));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        if (p >= M) continue;
        const int col = n0 + c0;
        if (!vec) {
#pragma unroll
            for (int q = 0; q < 16; q += 2) epi_store(e, g, p, col + q, __uint_as_float(v[q]), __uint_as_float(v[q + 1]));
            continue;
        }
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {  // two 8-channel chunks
            const int cc = col + 8 * hh;
            float f[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) f[q] = __uint_as_float(v[8 * hh + q]);
            bf16 *dst;
            if (e.kind == E_FWD) {
#pragma unroll
                for (int q = 0; q < 8; ++q) f[q] = fmaxf(f[q] + e.bias[cc + q], 0.0f);
                dst = e.out0 + cofs(prow, px, cc, e.ld0, g.W);
            } else if (cc < e.nsplit) {
                const uint4 mv = *reinterpret_cast<const uint4 *>(e.mask0 + cofs(prow, px, cc, e.ld0, g.W));
                const bf16 *m = reinterpret_cast<const bf16 *>(&mv);
#pragma unroll
                for (int q = 0; q < 8; ++q) f[q] = __bfloat162float(m[q]) > 0.0f ? f[q] : 0.0f;
                dst = e.out0 + cofs(prow, px, cc, e.ld0, g.W);
            } else {
                dst = e.out1 + cofs(prow, px, cc - e.nsplit, e.ld1, g.W);
            }
            __align__(16) bf162 hv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) hv[q] = __floats2bfloat162_rn(f[2 * q], f[2 * q + 1]);
            *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(hv);
        }
    }
}

template <int BN>
__global__ void __launch_bounds__(kTcThreads, 1) k_conv_tc(Gat g, const bf16 *__restrict__ B, int Kpad, size_t bz,
                                                          Epi e, int *err)
{
    pdl_entry();
    extern __shared__ __align__(1024) unsigned char smem[];
    using S = TcSmem<BN>;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char *bar_base = smem + kTcStages * S::kStage;
    const unsigned full0 = smem_u32(bar_base), empty0 = full0 + 8 * kTcStages, done = empty0 + 8 * kTcStages;
    unsigned *tmem_slot = reinterpret_cast<unsigned *>(bar_base + 8 * (2 * kTcStages + 1));
    const int M = g.N * g.H * g.W;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
    B += blockIdx.z * bz;
    const int KT = Kpad / kTcK;
    constexpr int kCols = BN < 32 ? 32 : BN;

    if (tid == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            mbar_init(full0 + 8 * s, 128);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const unsigned tmem = *tmem_slot;
    bool ok = true;

    if (warp < 4) {
        // ---- producers.  A: lane l of warp w stages rows 32 w + 8 s + (l & 7),
        // s = 0..3, chunks (l >> 3) and (l >> 3) + 4: one warp instruction reads
        // 8 pixels x 64 contiguous bytes.  B: BN / 16 chunks per thread, 4 rows
        // x 128 contiguous bytes per warp instruction ----
        const int hw = g.H * g.W, qh = lane >> 3;
        int rn[4], ri[4], rj[4];
        bool rv[4];
#pragma unroll
        for (int s4 = 0; s4 < 4; ++s4) {
            const int p = m0 + warp * 32 + 8 * s4 + (lane & 7);
            rv[s4] = p < M;
            const int n = rv[s4] ? p / hw : 0, r = p - n * hw;
            rn[s4] = n;
            ri[s4] = rv[s4] ? r / g.W : 0;
            rj[s4] = rv[s4] ? r - ri[s4] * g.W : 0;
        }
        int signalled = 0;
        for (int kt = 0; kt < KT && ok; ++kt) {
            const int s = kt % kTcStages;
            if (kt >= kTcStages) ok = mbar_wait(empty0 + 8 * s, ((kt / kTcStages) - 1) & 1);
            if (!ok) break;
            unsigned char *As = smem + s * S::kStage, *Bs = As + S::kA;
            const int k0 = kt * kTcK;
#pragma unroll
            for (int s4 = 0; s4 < 4; ++s4) {
                const int row = warp * 32 + 8 * s4 + (lane & 7);
                unsigned char *dst = As + ((row >> 3) * 8) * 128 + (row & 7) * 16;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int q = qh + 4 * h;
                    const bf16 *src = rv[s4] ? gat_src(g, rn[s4], ri[s4], rj[s4], k0 + q * 8) : nullptr;
                    cp16(dst + q * 128, src ? src : g.in0, src ? 16 : 0);
                }
            }
#pragma unroll
            for (int rr = 0; rr < BN / 16; ++rr) {
                const int c = tid + 128 * rr, nn = c >> 3, q = c & 7;
                cp16(Bs + ((nn >> 3) * 8 + q) * 128 + (nn & 7) * 16, B + (size_t)(n0 + nn) * Kpad + k0 + q * 8, 16);
            }
            cp_commit();
            if (kt >= kTcLag) {
                cp_wait<kTcLag>();
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                mbar_arrive(full0 + 8 * ((kt - kTcLag) % kTcStages));
                signalled = kt - kTcLag + 1;
            }
        }
        cp_wait<0>();
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        if (ok)
            for (int kt = signalled; kt < KT; ++kt) mbar_arrive(full0 + 8 * (kt % kTcStages));
    } else if (lane == 0) {
        // ---- MMA issuer ----
        constexpr unsigned idesc = umma_idesc<BN>();
        for (int kt = 0; kt < KT && ok; ++kt) {
            const int s = kt % kTcStages;
            ok = mbar_wait(full0 + 8 * s, (kt / kTcStages) & 1);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const unsigned a0 = smem_u32(smem + s * S::kStage), b0 = a0 + S::kA;
#pragma unroll
            for (int kk = 0; kk < kTcK / 16; ++kk) {
                const uint64_t ad = umma_desc(a0 + kk * 256), bd = umma_desc(b0 + kk * 256);
                const unsigned acc = (kt > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             empty0 + 8 * s)
                         : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(done)
                     : "memory");
        if (!mbar_wait(done, 0)) ok = false;  // no MMA in flight past this point
    }

    if (warp < 4) {
        // ---- epilogue: TMEM lanes 32 warp .. +31 are this warp's rows ----
        if (ok) ok = mbar_wait(done, 0);
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        tc_epilogue<BN>(e, g, tmem, m0, n0, M, warp, lane, __all_sync(0xffffffffu, ok));
    }
    if (!ok) atomicExch(err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 4) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kCols) : "memory");
    }
}

// ------------------------------------------------ tcgen05 halo convolution --
// A convolution whose CTA tile is 128 consecutive pixels of one output image
// row (n, i, x0 .. x0 + 127) by BN output channels, the accumulator in tensor
// memory.  The reduction runs in stages of CS input channels x one vertical
// tap: a stage holds the input row of that tap once, K-chunk by K-chunk (16
// bytes per pixel slot, the next chunk LBO bytes on), and the horizontal taps
// read it through descriptors whose start addresses differ by one slot (8-row
// groups 128 B apart).  Modes:
//   3x3 (stride 1, zero border): slots x0 - 1 .. x0 + 134 of input row i + ta - 1;
//   up: the same over the nearest-upsampled input (slot x reads pixel x / 2 of
//       row (i + ta - 1) / 2 of the half-resolution tensor);
//   down (2x2, stride 2): input row 2 i + ta, even pixels 2 (x0 + r) in slots
//       0 .. 127 and odd pixels in slots 128 .. 255, one array per horizontal tap.
// The stage's weights for all its horizontal taps arrive in one bulk copy,
// pre-packed in core-matrix order (k_pack_halo).
enum HaloMode { H_CONV3 = 0, H_UP3 = 1, H_DOWN2 = 2 };

struct Halo {
    const bf16 *in0, *in1;  // channels [0, c0) from in0, [c0, c0 + c1) from in1 (concatenation)
    int c0, c1;
    int N, H, W, xtiles;    // output image grid; 128-pixel tiles per image row
    int Hi, Wi;             // input tensor grid
    int mode, nst;          // HaloMode; stages: (c0 + c1) / CS x vertical taps
    int ncols;              // output channels (column tiles of BN)
};

template <int BN, int CS, bool DOWN>
struct HaloSmem {
    static constexpr int kSlots = DOWN ? 256 : 136;       // pixel slots per K-chunk (a multiple of 8)
    static constexpr int kLBO = (kSlots + 1) * 16;         // one padding slot: chunks fall in different banks
    static constexpr int kTH = DOWN ? 2 : 3;               // horizontal taps per stage
    static constexpr int kA = (CS / 8) * kLBO;
    static constexpr int kB = kTH * BN * CS * 2;
    static constexpr int kStage = kA + kB;
    static constexpr int kFit = (227 * 1024 - 512) / kStage;
    static constexpr int kStages = kFit >= 4 ? 4 : (kFit >= 2 ? kFit : 2);
    static constexpr int kBytes = kStages * kStage + 512;  // + barriers and the TMEM address
};

__device__ __forceinline__ uint64_t umma_desc_s(unsigned saddr, unsigned lbo, unsigned sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mbar_expect_tx(unsigned a, unsigned bytes)
{
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(a), "r"(bytes)
                 : "memory");
}

// Contiguous global -> shared bulk copy completing on an mbarrier (tx bytes).
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void *src, unsigned bytes, unsigned mbar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(mbar)
        : "memory");
}

// Persistent and warp-specialised: a CTA walks the tiles blockIdx.x,
// blockIdx.x + gridDim.x, ...; warps 0-3 stage operands through the stage ring
// (continuing across tiles), one thread of warp 8 issues the MMAs into one of
// two tensor-memory accumulator buffers, and warps 4-7 drain the other buffer
// (epilogue of tile t overlapping the loads and MMAs of tile t + 1).
constexpr int kPThreads = 288;  // warps 0-3 producers, 4-7 epilogue, 8 MMA issue

template <int BN, int CS, bool DOWN>
__global__ void __launch_bounds__(kPThreads, 1) k_conv_halo(Halo h, const bf16 *__restrict__ Bp, Epi e, int *err)
{
    pdl_entry();
    extern __shared__ __align__(1024) unsigned char smem[];
    using S = HaloSmem<BN, CS, DOWN>;
    constexpr int TH = S::kTH, TV = DOWN ? 2 : 3, NS = S::kStages, CH = CS / 8;
    // cp.async stages a producer keeps in flight before signalling: one stage of
    // slack between the MMA being waited for and the one being fed
    constexpr int LAG = NS >= 3 ? NS - 2 : 0;
    constexpr int kCols = DOWN ? 2 * BN : 4 * BN;  // two tile buffers (x two parities for the up mode)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char *bar_base = smem + NS * S::kStage;
    const unsigned full0 = smem_u32(bar_base), empty0 = full0 + 8 * NS;
    const unsigned accf0 = empty0 + 8 * NS, acce0 = accf0 + 16;  // accumulator full[2] / empty[2]
    unsigned *tmem_slot = reinterpret_cast<unsigned *>(bar_base + 8 * (2 * NS + 4));
    const bool up = !DOWN && h.mode == H_UP3;
    const int nacc = up ? 2 : 1;
    const int ntn = h.ncols / BN, ntiles = h.N * h.H * h.xtiles * ntn, KT = h.nst;

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(full0 + 8 * s, 129);  // 128 producers + the bulk copies' expect_tx arrival
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(accf0 + 8 * b, 1);
            mbar_init(acce0 + 8 * b, 128);
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 8) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const unsigned tmem = *tmem_slot;
    bool ok = true;

    // tile t: column tile nt (fastest), then 128-column tile xt of image row rowid
    auto decode = [&](int t, int &nt, int &rowid, int &x0) {
        nt = t % ntn;
        const int r = t / ntn;
        x0 = (r % h.xtiles) * kBM;
        rowid = r / h.xtiles;
    };

    if (warp < 4) {
        // ---- producers ----
        long long g = 0, sig = 0;  // stages staged / signalled by this thread
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            int nt, rowid, x0;
            decode(t, nt, rowid, x0);
            const int i = rowid % h.H, n = rowid / h.H;
            const bf16 *Bt = Bp + (size_t)nt * h.nst * TH * BN * CS;
            for (int kt = 0; kt < KT && ok; ++kt, ++g) {
                const int s = (int)(g % NS);
                if (g >= NS) ok = mbar_wait(empty0 + 8 * s, (unsigned)(((g / NS) - 1) & 1));
                if (!ok) break;
                unsigned char *As = smem + s * S::kStage, *Bs = As + S::kA;
                const int cc = kt / TV, ta = kt - TV * cc, cb = cc * CS;
                int y = DOWN ? 2 * i + ta : i + ta - 1;  // input row (output grid for the up mode)
                const bool row_ok = y >= 0 && y < (DOWN ? h.Hi : h.H);
                if (up) y >>= 1;
                const bf16 *tbase;
                int tC, coff;
                if (cb < h.c0) {
                    tbase = h.in0;
                    tC = h.c0;
                    coff = cb;
                } else {
                    tbase = h.in1;
                    tC = h.c1;
                    coff = cb - h.c0;
                }
                const size_t trow = (size_t)n * h.Hi + (row_ok ? y : 0);
                if (!DOWN) {
                    // slots x0 - 1 + sl of the input row: the columns inside [0, Wi)
                    // arrive by one bulk copy per channel chunk (a contiguous row
                    // segment of its plane), the others are zero
                    const int xs = max(x0 - 1, 0), xe = min(x0 - 1 + S::kSlots, h.Wi), s0 = xs - (x0 - 1);
                    if (tid == 0) {
                        const unsigned abytes = row_ok ? (unsigned)(xe - xs) * 16u * CH : 0u;
                        mbar_expect_tx(full0 + 8 * s, S::kB + abytes);
                        bulk_g2s(smem_u32(Bs), Bt + (size_t)kt * TH * BN * CS, S::kB, full0 + 8 * s);
                        if (row_ok)
                            for (int q = 0; q < CH; ++q)
                                bulk_g2s(smem_u32(As + q * S::kLBO + s0 * 16),
                                         tbase + cofs(trow, xs, coff + 8 * q, tC, h.Wi), (unsigned)(xe - xs) * 16u,
                                         full0 + 8 * s);
                    }
                    for (int idx = tid; idx < S::kSlots * CH; idx += 128) {
                        const int q = idx % CH, sl = idx / CH;
                        if (!(row_ok && sl >= s0 && sl < s0 + (xe - xs)))
                            *reinterpret_cast<uint4 *>(As + q * S::kLBO + sl * 16) = make_uint4(0u, 0u, 0u, 0u);
                    }
                    // only bulk copies (tracked by the byte count) and this thread's
                    // zero stores: signal at once
                    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                    mbar_arrive(full0 + 8 * s);
                    sig = g + 1;
                } else {
                    if (tid == 0) {
                        mbar_expect_tx(full0 + 8 * s, S::kB);
                        bulk_g2s(smem_u32(Bs), Bt + (size_t)kt * TH * BN * CS, S::kB, full0 + 8 * s);
                    }
                    for (int idx = tid; idx < S::kSlots * CH; idx += 128) {
                        const int q = idx % CH, sl = idx / CH;
                        const int r = sl & (kBM - 1), x = 2 * (x0 + r) + (sl >> 7);  // even / odd input pixels
                        const bool v = row_ok && x0 + r < h.W;
                        cp16(As + q * S::kLBO + sl * 16, v ? tbase + cofs(trow, x, coff + 8 * q, tC, h.Wi) : h.in0,
                             v ? 16 : 0);
                    }
                    cp_commit();
                    if (g >= LAG) {
                        cp_wait<LAG>();
                        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                        mbar_arrive(full0 + 8 * (int)((g - LAG) % NS));
                        sig = g - LAG + 1;
                    }
                }
            }
        }
        cp_wait<0>();
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        if (ok)
            for (; sig < g; ++sig) mbar_arrive(full0 + 8 * (int)(sig % NS));
    } else if (warp == 8) {
        if (lane == 0) {
            // ---- MMA issue: per stage TH taps x CS / 16 K-steps (x 2 parities for up) ----
            constexpr unsigned idesc = umma_idesc<BN>();
            long long g = 0;
            int lt = 0;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++lt) {
                const int buf = lt & 1;
                if (lt >= 2) ok = mbar_wait(acce0 + 8 * buf, (unsigned)(((lt >> 1) - 1) & 1));
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const unsigned acc0 = tmem + (unsigned)(buf * nacc * BN);
                for (int kt = 0; kt < KT && ok; ++kt, ++g) {
                    const int s = (int)(g % NS);
                    ok = mbar_wait(full0 + 8 * s, (unsigned)((g / NS) & 1));
                    if (!ok) break;
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    const unsigned a0 = smem_u32(smem + s * S::kStage), b0 = a0 + S::kA;
                    for (int b = 0; b < nacc; ++b)
#pragma unroll
                        for (int tb = 0; tb < TH; ++tb) {
                            // slot offset of the tap: tb (3x3), the even / odd input array
                            // (down), (b + tb + 1) / 2 (up: output column 2 (x0 + r) + b
                            // reads input column x0 + r + that - 1)
                            const int so = DOWN ? tb * kBM : (up ? (b + tb + 1) >> 1 : tb);
#pragma unroll
                            for (int kk = 0; kk < CS / 16; ++kk) {
                                const uint64_t ad = umma_desc_s(a0 + 2 * kk * S::kLBO + so * 16, S::kLBO, 128);
                                const uint64_t bd =
                                    umma_desc_s(b0 + tb * (BN * CS * 2) + 2 * kk * 128, 128, CH * 128);
                                const unsigned acc = (kt > 0 || tb > 0 || kk > 0) ? 1u : 0u;
                                asm volatile(
                                    "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                                        acc0 + (unsigned)(b * BN)),
                                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                                    : "memory");
                            }
                        }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                                     empty0 + 8 * s)
                                 : "memory");
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                                 accf0 + 8 * buf)
                             : "memory");
            }
            // no MMA in flight past this point (the last tile's commit completed)
            if (lt > 0 && !mbar_wait(accf0 + 8 * ((lt - 1) & 1), (unsigned)(((lt - 1) >> 1) & 1))) ok = false;
        }
    } else {
        // ---- epilogue (warps 4-7: TMEM lanes 32 (warp - 4) .. +31) ----
        const int ew = warp - 4;
        Gat g{};  // the epilogue needs only the output grid
        g.N = h.N;
        g.H = h.H;
        g.W = h.W;
        int lt = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++lt) {
            const int buf = lt & 1;
            const bool ok2 = ok && mbar_wait(accf0 + 8 * buf, (unsigned)((lt >> 1) & 1));
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const bool go = __all_sync(0xffffffffu, ok2);
            int nt, rowid, x0;
            decode(t, nt, rowid, x0);
            const int ps = up ? 2 : 1, nvalid = min(kBM, (up ? h.Wi : h.W) - x0);
            for (int b = 0; b < nacc; ++b) {
                const int m0 = rowid * h.W + ps * x0 + b;
                tc_epilogue<BN>(e, g, tmem + (unsigned)((buf * nacc + b) * BN), m0, nt * BN, m0 + ps * nvalid, ew,
                                lane, go, ps);
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            mbar_arrive(acce0 + 8 * buf);
            if (!go) {
                ok = false;
                break;
            }
        }
    }
    if (!ok) atomicExch(err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 8) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kCols) : "memory");
    }
}

// One tile per CTA (the schedule for the full-resolution layers with at most 32
// input channels per tensor, where many short tiles favour more resident CTAs
// over the persistent kernel's overlap): warps 0-3 stage and then run the
// epilogue, one thread of warp 4 issues the MMAs.
template <int BN, int CS, bool DOWN>
struct HaloSmem1 {
    using P = HaloSmem<BN, CS, DOWN>;
    static constexpr int kSlots = P::kSlots, kLBO = P::kLBO, kTH = P::kTH, kA = P::kA, kB = P::kB, kStage = P::kStage;
    static constexpr int kStages = kStage <= 40 * 1024 ? 4 : 3;
    static constexpr int kBytes = kStages * kStage + 256;
};

template <int BN, int CS, bool DOWN>
__global__ void __launch_bounds__(kTcThreads, 1) k_conv_halo1(Halo h, const bf16 *__restrict__ Bp, Epi e, int *err)
{
    pdl_entry();
    extern __shared__ __align__(1024) unsigned char smem[];
    using S = HaloSmem1<BN, CS, DOWN>;
    constexpr int TH = S::kTH, TV = DOWN ? 2 : 3;
    // cp.async stages a producer keeps in flight before signalling: one stage of
    // slack between the MMA being waited for and the one being fed
    constexpr int LAG = S::kStages - 2;
    constexpr int NS = S::kStages;
    constexpr int CH = CS / 8;  // 16-byte chunks per halo pixel
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char *bar_base = smem + NS * S::kStage;
    const unsigned full0 = smem_u32(bar_base), empty0 = full0 + 8 * NS, done = empty0 + 8 * NS;
    unsigned *tmem_slot = reinterpret_cast<unsigned *>(bar_base + 8 * (2 * NS + 1));
    // The tile: 128 columns from x0 of output row i -- of the input row for the up
    // mode, whose two accumulators hold the output columns 2 (x0 + r) + b, b = 0, 1
    // (each tap of either parity reads the half-resolution row one slot apart).
    const bool up = !DOWN && h.mode == H_UP3;
    const int xt = blockIdx.x % h.xtiles, rowid = blockIdx.x / h.xtiles;
    const int i = rowid % h.H, n = rowid / h.H, x0 = xt * kBM;
    const int nvalid = min(kBM, (up ? h.Wi : h.W) - x0);  // valid tile rows
    const int n0 = blockIdx.y * BN;
    const bf16 *Bt = Bp + (size_t)blockIdx.y * h.nst * TH * BN * CS;
    constexpr int kCols = DOWN ? (BN < 32 ? 32 : BN) : 2 * BN;  // the up mode's two accumulators

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(full0 + 8 * s, 129);  // 128 producers + the bulk copy's expect_tx arrival
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const unsigned tmem = *tmem_slot;
    bool ok = true;
    const int KT = h.nst;

    if (warp < 4) {
        // ---- producers: the halo row of the stage (8 consecutive threads read one
        // pixel's CS channels, 16 bytes each); thread 0 also issues the B bulk copy ----
        int signalled = 0;
        for (int kt = 0; kt < KT && ok; ++kt) {
            const int s = kt % NS;
            if (kt >= NS) ok = mbar_wait(empty0 + 8 * s, ((kt / NS) - 1) & 1);
            if (!ok) break;
            unsigned char *As = smem + s * S::kStage, *Bs = As + S::kA;
            const int cc = kt / TV, ta = kt - TV * cc, cb = cc * CS;
            int y = DOWN ? 2 * i + ta : i + ta - 1;  // input row (output grid for the up mode)
            const bool row_ok = y >= 0 && y < (DOWN ? h.Hi : h.H);
            if (h.mode == H_UP3) y >>= 1;
            const bf16 *tbase;
            int tC, coff;
            if (cb < h.c0) {
                tbase = h.in0;
                tC = h.c0;
                coff = cb;
            } else {
                tbase = h.in1;
                tC = h.c1;
                coff = cb - h.c0;
            }
            const size_t trow = (size_t)n * h.Hi + (row_ok ? y : 0);
            if (!DOWN) {
                // slots x0 - 1 + sl of the input row: the columns inside [0, Wi) arrive
                // by one bulk copy per channel chunk (a contiguous row segment of its
                // plane), the others are zero
                const int xs = max(x0 - 1, 0), xe = min(x0 - 1 + S::kSlots, h.Wi), s0 = xs - (x0 - 1);
                if (tid == 0) {
                    const unsigned abytes = row_ok ? (unsigned)(xe - xs) * 16u * CH : 0u;
                    mbar_expect_tx(full0 + 8 * s, S::kB + abytes);
                    bulk_g2s(smem_u32(Bs), Bt + (size_t)kt * TH * BN * CS, S::kB, full0 + 8 * s);
                    if (row_ok)
                        for (int q = 0; q < CH; ++q)
                            bulk_g2s(smem_u32(As + q * S::kLBO + s0 * 16), tbase + cofs(trow, xs, coff + 8 * q, tC, h.Wi),
                                     (unsigned)(xe - xs) * 16u, full0 + 8 * s);
                }
                for (int idx = tid; idx < S::kSlots * CH; idx += 128) {
                    const int q = idx % CH, sl = idx / CH;
                    if (!(row_ok && sl >= s0 && sl < s0 + (xe - xs)))
                        *reinterpret_cast<uint4 *>(As + q * S::kLBO + sl * 16) = make_uint4(0u, 0u, 0u, 0u);
                }
            } else {
                if (tid == 0) {
                    mbar_expect_tx(full0 + 8 * s, S::kB);
                    bulk_g2s(smem_u32(Bs), Bt + (size_t)kt * TH * BN * CS, S::kB, full0 + 8 * s);
                }
                for (int idx = tid; idx < S::kSlots * CH; idx += 128) {
                    const int q = idx % CH, sl = idx / CH;
                    const int r = sl & (kBM - 1), x = 2 * (x0 + r) + (sl >> 7);  // even / odd input pixels
                    const bool v = row_ok && x0 + r < h.W;
                    cp16(As + q * S::kLBO + sl * 16, v ? tbase + cofs(trow, x, coff + 8 * q, tC, h.Wi) : h.in0,
                         v ? 16 : 0);
                }
            }
            if (!DOWN) {
                // only bulk copies (tracked by the barrier's byte count) and zero
                // stores of this thread: signal at once
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                mbar_arrive(full0 + 8 * s);
                signalled = kt + 1;
            } else {
                cp_commit();
                if (kt >= LAG) {
                    cp_wait<LAG>();
                    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                    mbar_arrive(full0 + 8 * ((kt - LAG) % NS));
                    signalled = kt - LAG + 1;
                }
            }
        }
        cp_wait<0>();
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        if (ok)
            for (int kt = signalled; kt < KT; ++kt) mbar_arrive(full0 + 8 * (kt % NS));
    } else if (lane == 0) {
        // ---- MMA issuer: per stage TH taps x CS / 16 K-steps ----
        constexpr unsigned idesc = umma_idesc<BN>();
        for (int kt = 0; kt < KT && ok; ++kt) {
            const int s = kt % NS;
            ok = mbar_wait(full0 + 8 * s, (kt / NS) & 1);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const unsigned a0 = smem_u32(smem + s * S::kStage), b0 = a0 + S::kA;
            for (int b = 0; b < (up ? 2 : 1); ++b)
#pragma unroll
                for (int tb = 0; tb < TH; ++tb) {
                    // slot offset of the tap: tb (3x3), the even / odd input array (down),
                    // (b + tb + 1) / 2 (up: output column 2 (x0 + r) + b reads input x0 + r + that - 1)
                    const int so = DOWN ? tb * kBM : (up ? (b + tb + 1) >> 1 : tb);
#pragma unroll
                    for (int kk = 0; kk < CS / 16; ++kk) {
                        const uint64_t ad = umma_desc_s(a0 + 2 * kk * S::kLBO + so * 16, S::kLBO, 128);
                        const uint64_t bd = umma_desc_s(b0 + tb * (BN * CS * 2) + 2 * kk * 128, 128, CH * 128);
                        const unsigned acc = (kt > 0 || tb > 0 || kk > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + b * BN),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                            : "memory");
                    }
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             empty0 + 8 * s)
                         : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(done)
                     : "memory");
        if (!mbar_wait(done, 0)) ok = false;  // no MMA in flight past this point
    }

    if (warp < 4) {
        if (ok) ok = mbar_wait(done, 0);
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        Gat g{};  // the epilogue needs only the output grid
        g.N = h.N;
        g.H = h.H;
        g.W = h.W;
        const bool go = __all_sync(0xffffffffu, ok);
        for (int b = 0; b < (up ? 2 : 1); ++b) {
            const int ps = up ? 2 : 1, m0 = rowid * h.W + ps * x0 + b;
            tc_epilogue<BN>(e, g, tmem + b * BN, m0, n0, m0 + ps * nvalid, warp, lane, go, ps);
        }
    }
    if (!ok) atomicExch(err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 4) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kCols) : "memory");
    }
}


// Weight gradient: part[z][k][n] = sum over the rows p of split z of A(p, k)
// G[p][n] for the weight rows [blockIdx.x kBM, +kBM) and columns [blockIdx.y BN,
// +BN).  A(p, k) is the layer's forward gather; rows are taken kBK at a time.
template <int BN>
__global__ void __launch_bounds__(kGT) k_wgrad(Gat g, const bf16 *__restrict__ G, int ldg, int chunks_per_split,
                                               int Kpad, float *__restrict__ part)
{
    pdl_entry();
    constexpr int AS = kBM + 8;
    constexpr int BS = BN + 8;
    constexpr int WN = BN / 2;
    constexpr int NT = WN / 8;
    __shared__ __align__(128) bf16 As[kStages][kBK][AS];  // [pixel][weight row]
    __shared__ __align__(128) bf16 Bs[kStages][kBK][BS];  // [pixel][channel]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 3, wn = warp >> 2;
    const int M = g.N * g.H * g.W, hw = g.H * g.W;
    const int k0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
    const int nchunks = (M + kBK - 1) / kBK;
    const int c_begin = blockIdx.z * chunks_per_split;
    const int c_end = min(c_begin + chunks_per_split, nchunks);
    const int br = tid / (BN / 8), bc = tid % (BN / 8);

    auto load = [&](int stage, int chunk) {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int q = tid + kGT * s, row = q >> 4, kcol = q & 15;
            const int p = chunk * kBK + row;
            const bf16 *src = nullptr;
            if (p < M) {
                const int n = p / hw, r = p - n * hw, i = r / g.W, j = r - i * g.W;
                src = gat_src(g, n, i, j, k0 + kcol * 8);
            }
            cp16(&As[stage][row][kcol * 8], src ? src : g.in0, src ? 16 : 0);
        }
        if (br < kBK) {
            const int p = chunk * kBK + br;
            const bf16 *src = G;
            if (p < M) {
                const size_t prow = (size_t)(p / g.W);
                src = G + cofs(prow, p - (int)prow * g.W, n0 + bc * 8, ldg, g.W);
            }
            cp16(&Bs[stage][br][bc * 8], src, p < M ? 16 : 0);
        }
    };

    float acc[2][NT][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < NT; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.0f;

    const int KT = max(c_end - c_begin, 0);
#pragma unroll
    for (int s = 0; s < kStages - 1; ++s) {
        if (s < KT) load(s, c_begin + s);
        cp_commit();
    }
    for (int kt = 0; kt < KT; ++kt) {
        cp_wait<kStages - 2>();
        __syncthreads();
        {
            const int nk = kt + kStages - 1;
            if (nk < KT) load(nk % kStages, c_begin + nk);
            cp_commit();
        }
        const int st = kt % kStages;
#pragma unroll
        for (int kk = 0; kk < kBK; kk += 16) {
            unsigned a[2][4], b[NT][2];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
                ldm_x4_t(a[mt], &As[st][kk + (lane & 7) + ((lane >> 4) << 3)][wm * 32 + mt * 16 + ((lane >> 3) & 1) * 8]);
#pragma unroll
            for (int np = 0; np < NT / 2; ++np) {
                unsigned r[4];
                ldm_x4_t(r, &Bs[st][kk + (lane & 15)][wn * WN + np * 16 + (lane >> 4) * 8]);
                b[2 * np][0] = r[0];
                b[2 * np][1] = r[1];
                b[2 * np + 1][0] = r[2];
                b[2 * np + 1][1] = r[3];
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) mma16816(acc[mt][nt], a[mt], b[nt]);
        }
    }
    cp_wait<0>();

    const int ldp = gridDim.y * BN;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = k0 + wm * 32 + mt * 16 + (lane >> 2) + 8 * h;
                const int col = n0 + wn * WN + nt * 8 + 2 * (lane & 3);
                *reinterpret_cast<float2 *>(part + ((size_t)blockIdx.z * Kpad + k) * ldp + col) =
                    make_float2(acc[mt][nt][2 * h], acc[mt][nt][2 * h + 1]);
            }
}

// ------------------------------------------------------------ small kernels --
constexpr int kT = 256;
constexpr int kHeadVals = 34;  // per-block partials of the head: dw[32], db, loss

// x FP32 [M][2] (pixel p = row W + x) -> chunk-planar BF16 with kInPad channels, channels 2.. zero.
__global__ void k_input(const float *__restrict__ x, long long M, int W, bf16 *__restrict__ xin)
{
    pdl_entry();
    const long long p = blockIdx.x * (long long)kT + threadIdx.x;
    if (p >= M) return;
    const size_t prow = (size_t)(p / W);
    const int px = (int)(p - (long long)prow * W);
    const float2 v = *reinterpret_cast<const float2 *>(x + 2 * p);
    __align__(16) bf16 row[kInPad];
    row[0] = __float2bfloat16_rn(v.x);
    row[1] = __float2bfloat16_rn(v.y);
#pragma unroll
    for (int c = 2; c < kInPad; ++c) row[c] = __float2bfloat16_rn(0.0f);
#pragma unroll
    for (int q = 0; q < kInPad / 8; ++q)
        *reinterpret_cast<uint4 *>(xin + cofs(prow, px, 8 * q, kInPad, W)) = reinterpret_cast<const uint4 *>(row)[q];
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// 1x1 FP32 head over the 32-channel tensor a: out = a . w + b.  With a target
// (training): dout = 2 (out - t) / M, the gradient of the head input's
// pre-activation G = bf16(dout w * (a > 0)), and per-block partials of dw, db and
// the squared error (kHeadVals per block).
__global__ void __launch_bounds__(kT) k_head(const bf16 *__restrict__ a, const float *__restrict__ w, long long M,
                                             int W, float *__restrict__ out, const float *__restrict__ target,
                                             float inv_m, bf16 *__restrict__ G, float *__restrict__ part)
{
    pdl_entry();
    __shared__ float sh[kT / 32][kHeadVals];
    const long long p = blockIdx.x * (long long)kT + threadIdx.x;
    float av[32];
    float o = 0.0f;
    const size_t prow = (size_t)(p / W);
    const int px = (int)(p - (long long)prow * W);
    if (p < M) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint4 u = *reinterpret_cast<const uint4 *>(a + cofs(prow, px, 8 * q, 32, W));
            const bf16 *h = reinterpret_cast<const bf16 *>(&u);
#pragma unroll
            for (int c = 0; c < 8; ++c) av[8 * q + c] = __bfloat162float(h[c]);
        }
        o = w[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) o = fmaf(av[c], w[c], o);
        out[p] = o;
    }
    if (!target) return;
    float d = 0.0f, se = 0.0f;
    if (p < M) {
        const float r = o - target[p];
        d = 2.0f * r * inv_m;
        se = r * r;
        __align__(16) bf16 g[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) g[c] = __float2bfloat16_rn(av[c] > 0.0f ? d * w[c] : 0.0f);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            *reinterpret_cast<uint4 *>(G + cofs(prow, px, 8 * q, 32, W)) = reinterpret_cast<const uint4 *>(g)[q];
    } else {
#pragma unroll
        for (int c = 0; c < 32; ++c) av[c] = 0.0f;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        const float s = warp_sum(d * av[c]);
        if (lane == 0) sh[warp][c] = s;
    }
    {
        const float s = warp_sum(d);
        if (lane == 0) sh[warp][32] = s;
        const float q = warp_sum(se);
        if (lane == 0) sh[warp][33] = q;
    }
    __syncthreads();
    if (threadIdx.x < kHeadVals) {
        float s = 0.0f;
        for (int wv = 0; wv < kT / 32; ++wv) s += sh[wv][threadIdx.x];
        part[(size_t)blockIdx.x * kHeadVals + threadIdx.x] = s;
    }
}

// Head gradient and loss from the per-block partials (fixed order).
__global__ void k_head_final(const float *__restrict__ part, int nblocks, float *__restrict__ gw, double *loss,
                             double inv_m)
{
    pdl_entry();
    const int v = threadIdx.x;
    if (v >= kHeadVals) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[(size_t)b * kHeadVals + v];
    if (v < 33)
        gw[v] = (float)s;
    else
        *loss = s * inv_m;
}

// Input gradient of an upsampling layer: G(n, i, j, c) = bf16(sum of the 2x2
// block of tmp (full grid, NHWC FP32) * (low > 0)), low the half-grid input
// tensor; G and low chunk-planar, the thread index running in their order.
__global__ void k_up_pool(const float *__restrict__ tmp, const bf16 *__restrict__ low, int N, int h, int w, int C,
                          bf16 *__restrict__ G)
{
    pdl_entry();
    const long long k = blockIdx.x * (long long)kT + threadIdx.x;
    const long long total = (long long)N * h * w * C;
    if (k >= total) return;
    const int c8 = (int)(k & 7);
    const long long t = k >> 3;
    const int j = (int)(t % w);
    const long long t2 = t / w;
    const int q = (int)(t2 % (C / 8));
    const long long row = t2 / (C / 8);
    const int i = (int)(row % h), n = (int)(row / h), c = 8 * q + c8;
    const size_t W2 = 2 * (size_t)w;
    const size_t o = (((size_t)n * 2 * h + 2 * i) * W2 + 2 * j) * C + c;
    const float s = (tmp[o] + tmp[o + C]) + (tmp[o + W2 * C] + tmp[o + W2 * C + C]);
    G[k] = __float2bfloat16_rn(__bfloat162float(low[k]) > 0.0f ? s : 0.0f);
}

// Column sums of a chunk-planar G [rows][C / 8][W][8] (bias gradient): block b
// sums rows [b rpb, (b + 1) rpb) into part[b][C].  Thread t always meets
// channel 8 q + t % 8 of chunk q (kT is a multiple of 8).
__global__ void __launch_bounds__(kT) k_colsum(const bf16 *__restrict__ G, int rows, int W, int C, int rpb,
                                               float *__restrict__ part)
{
    pdl_entry();
    __shared__ float sh[32][kT];  // C / 8 <= 32 chunks
    const int nq = C / 8;
    float acc[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) acc[q] = 0.0f;
    const int r0 = blockIdx.x * rpb, r1 = min(r0 + rpb, rows);
    for (int r = r0; r < r1; ++r)
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            if (q >= nq) break;
            const bf16 *seg = G + ((size_t)r * nq + q) * (size_t)W * 8;
            for (int idx = threadIdx.x; idx < W * 8; idx += kT) acc[q] += __bfloat162float(seg[idx]);
        }
#pragma unroll
    for (int q = 0; q < 32; ++q)
        if (q < nq) sh[q][threadIdx.x] = acc[q];
    __syncthreads();
    if (threadIdx.x < C) {
        const int q = threadIdx.x >> 3, c8 = threadIdx.x & 7;
        float s = 0.0f;
        for (int t = c8; t < kT; t += 8) s += sh[q][t];
        part[(size_t)blockIdx.x * C + threadIdx.x] = s;
    }
}

__global__ void k_colsum_final(const float *__restrict__ part, int nblocks, int C, float *__restrict__ gb)
{
    pdl_entry();
    const int c = blockIdx.x * kT + threadIdx.x;
    if (c >= C) return;
    float s = 0.0f;
    for (int b = 0; b < nblocks; ++b) s += part[(size_t)b * C + c];
    gb[c] = s;
}

// Weight gradient of a layer from the split partials: gw[(t ci + c) co + o] =
// sum_z part[z][t cinp + c][o], in split order.
__global__ void k_wgrad_reduce(const float *__restrict__ part, int splits, int Kpad, int co, int cinp, int ci,
                               int ntaps, float *__restrict__ gw)
{
    pdl_entry();
    const long long idx = blockIdx.x * (long long)kT + threadIdx.x;
    const long long total = (long long)ntaps * ci * co;
    if (idx >= total) return;
    const int o = (int)(idx % co);
    const long long r = idx / co;
    const int c = (int)(r % ci), t = (int)(r / ci);
    const int k = t * cinp + c;
    float s = 0.0f;
    for (int z = 0; z < splits; ++z) s += part[((size_t)z * Kpad + k) * co + o];
    gw[idx] = s;
}

// Adam with bias correction (b1t = 1 - beta1^t, b2t = 1 - beta2^t).
__global__ void k_adam(float *__restrict__ th, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, long long n, float lr, float b1t, float b2t)
{
    pdl_entry();
    const long long k = blockIdx.x * (long long)kT + threadIdx.x;
    if (k >= n) return;
    const float gk = g[k];
    const float mk = 0.9f * m[k] + 0.1f * gk;
    const float vk = 0.999f * v[k] + 0.001f * gk * gk;
    m[k] = mk;
    v[k] = vk;
    th[k] -= lr * (mk / b1t) / (sqrtf(vk / b2t) + 1e-8f);
}

// Halo-ordered BF16 weights of a halo GEMM: for each column tile nt (BN wide),
// stage (cc, ta) and horizontal tap tb (tv x th taps, tap t = th ta + tb), a
// BN x CS block in core-matrix order: element (n, ch) at
// ((n / 8) (CS / 8) + ch / 8) 64 + (n % 8) 8 + ch % 8.  Forward (flip = 0):
// value W[t][cc CS + ch][nt BN + n] (zero for channels >= ci, the input
// layer's padding); 3x3 input gradient (flip = 1): W[8 - t][nt BN + n][cc CS + ch].
// W is [tv th][ci][co] FP32.
__global__ void k_pack_halo(const float *__restrict__ W, int ci, int co, int kin, int ncols, int BN, int CS, int tv,
                            int th, int flip, bf16 *__restrict__ out)
{
    pdl_entry();
    const long long idx = blockIdx.x * (long long)kT + threadIdx.x;
    const long long nst = (long long)(kin / CS) * tv;
    const long long blk = (long long)BN * CS;
    if (idx >= (long long)(ncols / BN) * nst * th * blk) return;
    const long long b = idx / blk;
    const int w = (int)(idx - b * blk);
    const int tb = (int)(b % th), st = (int)((b / th) % nst), nt = (int)(b / (th * nst));
    const int cc = st / tv, ta = st - tv * cc;
    const int rb = w / 64, r = w - rb * 64, nb = rb / (CS / 8), qb = rb - nb * (CS / 8);
    const int nn = nb * 8 + r / 8, ch = qb * 8 + r % 8;
    const int col = nt * BN + nn, kc = cc * CS + ch, t = th * ta + tb;
    float v;
    if (!flip)
        v = kc < ci ? W[((size_t)t * ci + kc) * co + col] : 0.0f;
    else
        v = W[((size_t)(8 - t) * ci + col) * co + kc];
    out[idx] = __float2bfloat16_rn(v);
}

// BF16 copy of a stride-2 layer's weights W [4][ci][co]: the K-major matrices
// [t][c][o] of its input-gradient GEMMs (one per sub-pixel t).
__global__ void k_pack_down(const float *__restrict__ W, long long n, bf16 *__restrict__ Bk)
{
    pdl_entry();
    const long long q = blockIdx.x * (long long)kT + threadIdx.x;
    if (q < n) Bk[q] = __float2bfloat16_rn(W[q]);
}

// ------------------------------------------------- features of a pressure problem --
// part[b] = sum of b^2 over block b's cells (FP64).
__global__ void __launch_bounds__(kT) k_feat_bsum(const double *__restrict__ b, int n, double *__restrict__ part)
{
    pdl_entry();
    __shared__ double sh[kT / 32];
    double s = 0.0;
    for (int c = blockIdx.x * kT + threadIdx.x; c < n; c += gridDim.x * kT) s += b[c] * b[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kT / 32; ++w) t += sh[w];
        part[blockIdx.x] = t;
    }
}

// Sum of n partials, computed once per block (warp 0, fixed order) and shared:
// the same value in every block.  Call from all threads of the block.
__device__ double block_sum_parts(const double *part, int n)
{
    __shared__ double r;
    if (threadIdx.x < 32) {
        double s = 0.0;
        for (int k = threadIdx.x; k < n; k += 32) s += part[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) r = s;
    }
    __syncthreads();
    const double v = r;
    __syncthreads();  // r may be written again by the next call
    return v;
}

__device__ __forceinline__ double cell_beta(const double *bu, const double *bv, int nx, int i, int j)
{
    return 0.25 * (bu[j * (nx + 1) + i] + bu[j * (nx + 1) + i + 1] + bv[j * nx + i] + bv[(j + 1) * nx + i]);
}

// Features x [n][2] (and, if phi is given, the target t [n]) of A phi = b.
__global__ void k_features(int nx, int ny, const double *__restrict__ b, const double *__restrict__ bu,
                           const double *__restrict__ bv, const double *__restrict__ inp, double rho_w,
                           const double *__restrict__ part, int nparts, const double *__restrict__ phi,
                           float *__restrict__ x, float *__restrict__ t)
{
    pdl_entry();
    const double s2 = block_sum_parts(part, nparts);
    const int c = blockIdx.x * kT + threadIdx.x;
    if (c >= nx * ny) return;
    const int i = c % nx, j = c / nx;
    const double beta = cell_beta(bu, bv, nx, i, j);
    float x0 = 0.0f, x1 = 0.0f, tt = 0.0f;
    if (s2 > 0.0 && beta > 0.0) {  // FP32 arithmetic: the features are FP32 network inputs
        const float irms = (float)(1.0 / sqrt(s2 / (double(nx) * ny)));
        x0 = (float)b[c] * irms;
        x1 = 0.25f * logf((float)(rho_w * beta) / (float)inp[0]);
        if (phi) tt = (float)phi[c] * (float)beta * irms;
    }
    *reinterpret_cast<float2 *>(x + 2 * (size_t)c) = make_float2(x0, x1);
    if (phi) t[c] = tt;
}

// phi0 = out rms(b) / beta_c; then part2[b] = sum of (b - A phi0)^2 over block b.
__global__ void k_guess(int nx, int ny, const double *__restrict__ b, const double *__restrict__ bu,
                        const double *__restrict__ bv, const double *__restrict__ part, int nparts,
                        const float *__restrict__ out, double *__restrict__ phi)
{
    pdl_entry();
    const double s2 = block_sum_parts(part, nparts);
    const int c = blockIdx.x * kT + threadIdx.x;
    if (c >= nx * ny) return;
    const int i = c % nx, j = c / nx;
    const double beta = cell_beta(bu, bv, nx, i, j);
    const float rms = (float)sqrt(s2 / (double(nx) * ny));  // FP32: an initial guess, judged by its FP64 residual
    phi[c] = (s2 > 0.0 && beta > 0.0) ? double(out[c] * rms / (float)beta) : 0.0;
}

__global__ void __launch_bounds__(kT) k_guess_resid(int nx, int ny, const double *__restrict__ b,
                                                    const double *__restrict__ bu, const double *__restrict__ bv,
                                                    const double *__restrict__ phi, double *__restrict__ part)
{
    pdl_entry();
    __shared__ double sh[kT / 32];
    double s = 0.0;
    for (int c = blockIdx.x * kT + threadIdx.x; c < nx * ny; c += gridDim.x * kT) {
        const int i = c % nx, j = c / nx;
        const double r = b[c] - (diag_at(bu, bv, nx, ny, i, j) * phi[c] - offsum_at(bu, bv, phi, nx, ny, i, j));
        s += r * r;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kT / 32; ++w) t += sh[w];
        part[blockIdx.x] = t;
    }
}

// Keep phi0 only if ||b - A phi0|| < ||b|| (else phi0 = 0); count tried / kept.
__global__ void k_guess_select(int n, const double *__restrict__ pb, const double *__restrict__ pr, int nparts,
                               double *__restrict__ phi, long long *stats)
{
    pdl_entry();
    const double b2 = block_sum_parts(pb, nparts);
    const double r2 = block_sum_parts(pr, nparts);
    const bool keep = r2 < b2;
    const int c = blockIdx.x * kT + threadIdx.x;
    if (!keep && c < n) phi[c] = 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        stats[0] += 1;
        stats[1] += keep ? 1 : 0;
    }
}

}  // namespace
}  // namespace wec

struct wec_net {
    int H = 0, W = 0, maxb = 0;
    cudaStream_t st = nullptr;
    size_t nparam = 0;
    float *theta = nullptr, *grad = nullptr, *am = nullptr, *av = nullptr;  // FP32 [nparam] each
    long long adam_t = 0;
    bool wdirty = true;                       // BF16 matrices older than theta
    bf16 *wmat = nullptr;                     // every layer's BF16 matrices
    size_t flat[wec::kNumLayers] = {};        // layer weights in theta (bias follows)
    size_t wb[wec::kNumLayers] = {};          // stride-2 layers: input-gradient matrices in wmat
    size_t hf[wec::kNumLayers] = {}, hb[wec::kNumLayers] = {};  // halo-ordered 3x3 matrices (forward / input gradient)
    int bnf[wec::kNumLayers] = {}, bnb[wec::kNumLayers] = {};   // their column-tile widths
    bf16 *xin = nullptr;                      // [maxb][H][W][8]
    bf16 *act[wec::kNumLayers] = {};          // layer outputs
    float *out = nullptr;                     // [maxb][H][W]
    bf16 *gA[4] = {}, *gB[4] = {}, *skip[3] = {};  // gradients per level
    float *tmpf = nullptr;                    // input gradient of an upsampling layer (full grid)
    float *part = nullptr;                    // split-K partials of the weight gradients
    size_t part_n = 0;
    float *cpart = nullptr;                   // column-sum / head partials
    float *xb = nullptr, *tb = nullptr;       // gathered batch (or a tank's features)
    double *loss = nullptr, *lossh = nullptr; // device / pinned host
    double *dpart = nullptr;                  // FP64 partials of the tank guess (2 x kRedBlocks)
    int *err = nullptr;                       // device: set when a tensor-core pipeline wait expired
    std::vector<void *> allocs;
};

namespace wec {
namespace {

constexpr int kCsumBlocks = 304;
constexpr int kWgradTarget = 608;  // CTAs a weight-gradient launch aims for (4 per SM)

int ilog2(int v)
{
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

size_t weight_count(int L) { return (size_t)taps(kLayers[L].kind) * kLayers[L].ci * kLayers[L].co; }
int fwd_K(int L) { return taps(kLayers[L].kind) * cin_pad(kLayers[L].ci); }
int level_h(const wec_net *N, int l) { return N->H >> l; }
int level_w(const wec_net *N, int l) { return N->W >> l; }
int chans(int l) { return 32 << l; }

void layer_inputs(const wec_net *N, int L, const bf16 **in0, const bf16 **in1)
{
    *in1 = nullptr;
    for (int l = 0; l < 4; ++l) {
        if (L == enc_a(l)) *in0 = l == 0 ? N->xin : N->act[down(l - 1)];
        if (L == enc_b(l)) *in0 = N->act[enc_a(l)];
        if (l < 3 && L == down(l)) *in0 = N->act[enc_b(l)];
        if (l < 3 && L == up(l)) *in0 = l == 2 ? N->act[enc_b(3)] : N->act[dec(l + 1)];
        if (l < 3 && L == cat(l)) {
            *in0 = N->act[up(l)];
            *in1 = N->act[enc_b(l)];
        }
        if (l < 3 && L == dec(l)) *in0 = N->act[cat(l)];
    }
}

// The forward gather of layer L (its input tensors, output grid of its level).
Gat fwd_gather(const wec_net *N, int L, int batch)
{
    const LayerDef &d = kLayers[L];
    const int cinp = cin_pad(d.ci), H = level_h(N, d.level), W = level_w(N, d.level);
    Gat g{};
    layer_inputs(N, L, &g.in0, &g.in1);
    g.c0 = g.in1 ? cinp / 2 : cinp;
    g.c1 = g.in1 ? cinp / 2 : 0;
    g.lcin = ilog2(cinp);
    g.kind = d.kind == L_CONV3 ? G_CONV3 : (d.kind == L_UP3 ? G_UP3 : G_DOWN2);
    g.N = batch;
    g.H = H;
    g.W = W;
    g.Hi = d.kind == L_UP3 ? H / 2 : (d.kind == L_DOWN2 ? 2 * H : H);
    g.Wi = d.kind == L_UP3 ? W / 2 : (d.kind == L_DOWN2 ? 2 * W : W);
    g.K = fwd_K(L);
    return g;
}


template <int BN>
int launch_tc(cudaStream_t st, dim3 grid, const Gat &g, const bf16 *B, int Kpad, size_t bz, const Epi &e, int *err)
{
    static bool attr = false;  // dynamic shared memory above 48 KB, set once per instantiation
    if (!attr) {
        WEC_CK(cudaFuncSetAttribute(k_conv_tc<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcSmem<BN>::kBytes));
        attr = true;
    }
    WEC_CK(launch_k(k_conv_tc<BN>, grid, kTcThreads, TcSmem<BN>::kBytes, st, g, B, Kpad, bz, e, err));
    return WEC_OK;
}

// One convolution GEMM on the tensor cores: B is the K-major weight matrix
// (ncols rows of Kpad elements; blockIdx.z selects one bz elements further on).
// Tile width: the widest of 256/128/64/32 dividing ncols that still gives >= 256
// CTAs (about two per SM), else 32.  tag: the layer index (forward) or 100 +
// layer (input gradient), reported as the profile level of the launch.
int gemm(wec_net *N, cudaStream_t st, int tag, const Gat &g, const bf16 *B, int Kpad, size_t bz, int ncols, int nz,
         const Epi &e)
{
    const long long M = (long long)g.N * g.H * g.W;
    const long long mt = (M + kBM - 1) / kBM;
    int bn = 32;
    for (int c : {256, 128, 64})
        if (ncols % c == 0 && mt * (ncols / c) * nz >= 256) {
            bn = c;
            break;
        }
    dim3 grid((unsigned)mt, (unsigned)(ncols / bn), (unsigned)nz);
    WEC_PROF("net_conv", tag, 2.0 * M * nz * ((double)(g.c0 + g.c1) + ncols) + 2.0 * Kpad * ncols * nz, st);
    switch (bn) {
    case 256: return launch_tc<256>(st, grid, g, B, Kpad, bz, e, N->err);
    case 128: return launch_tc<128>(st, grid, g, B, Kpad, bz, e, N->err);
    case 64: return launch_tc<64>(st, grid, g, B, Kpad, bz, e, N->err);
    default: return launch_tc<32>(st, grid, g, B, Kpad, bz, e, N->err);
    }
}

// ---- convolutions with the halo kernel ----
inline int halo_cs(int c) { return c >= 64 ? 64 : c; }  // channels per stage (c: channels of one input tensor)
inline bool halo_fwd(int L) { return kLayers[L].kind != L_HEAD; }
inline bool halo_bwd(int L) { return L != enc_a(0) && (kLayers[L].kind == L_CONV3 || kLayers[L].kind == L_UP3); }
inline int halo_kin(int L, bool bwd) { return bwd ? kLayers[L].co : cin_pad(kLayers[L].ci); }
inline int halo_mode(int kind) { return kind == L_UP3 ? H_UP3 : (kind == L_DOWN2 ? H_DOWN2 : H_CONV3); }

// Column-tile width: the widest of 128 / 64 dividing ncols that still gives >= 128
// tiles for one image (measured: wider tiles beat more, narrower ones down to
// about one tile per SM), else 32.  The up mode tiles the half-resolution row.
int halo_bn(const wec_net *N, int level, int ncols, bool up = false)
{
    const int w = up ? level_w(N, level) / 2 : level_w(N, level);
    const long long tiles = (long long)level_h(N, level) * ((w + kBM - 1) / kBM);
    for (int c : {128, 64})
        if (ncols % c == 0 && tiles * (ncols / c) >= 128) return c;
    return 32;
}

// Persistent grid: as many CTAs as fit on the GPU at once (shared memory and
// tensor-memory columns), at most one per tile.
template <int BN, int CS, bool DOWN>
int launch_halo_t(cudaStream_t st, long long ntiles, const Halo &h, const bf16 *B, const Epi &e, int *err)
{
    using S = HaloSmem<BN, CS, DOWN>;
    static int ctas = 0;  // resident CTAs on the device, computed once per instantiation
    if (!ctas) {
        WEC_CK(cudaFuncSetAttribute(k_conv_halo<BN, CS, DOWN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    S::kBytes));
        int dev = 0, sms = 0, occ = 0;
        WEC_CK(cudaGetDevice(&dev));
        WEC_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        WEC_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_conv_halo<BN, CS, DOWN>, kPThreads, S::kBytes));
        const int cols = DOWN ? 2 * BN : 4 * BN;
        ctas = sms * std::max(1, std::min(occ, 512 / cols));
    }
    const unsigned grid = (unsigned)std::min<long long>(ntiles, ctas);
    WEC_CK(launch_k(k_conv_halo<BN, CS, DOWN>, grid, kPThreads, S::kBytes, st, h, B, e, err));
    return WEC_OK;
}

// One tile per CTA (k_conv_halo1): grid (image rows x column tiles of 128, column tiles of BN).
template <int BN, int CS>
int launch_halo1_t(cudaStream_t st, const Halo &h, const bf16 *B, const Epi &e, int *err)
{
    using S = HaloSmem1<BN, CS, false>;
    static bool attr = false;  // dynamic shared memory above 48 KB, set once per instantiation
    if (!attr) {
        WEC_CK(cudaFuncSetAttribute(k_conv_halo1<BN, CS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    S::kBytes));
        attr = true;
    }
    dim3 grid((unsigned)(h.N * h.H * h.xtiles), (unsigned)(h.ncols / BN));
    WEC_CK(launch_k(k_conv_halo1<BN, CS, false>, grid, kTcThreads, S::kBytes, st, h, B, e, err));
    return WEC_OK;
}

template <int BN>
int launch_halo_cs(int CS, bool down, cudaStream_t st, long long ntiles, const Halo &h, const bf16 *B, const Epi &e,
                   int *err)
{
    // schedule: layers with at most 32 input channels per tensor (full resolution:
    // many short tiles) one tile per CTA; the others persistent
    if (!down && CS == 32) return launch_halo1_t<BN, 32>(st, h, B, e, err);
    if (!down && CS == 16) return launch_halo1_t<BN, 16>(st, h, B, e, err);
    if (down) {
        if (CS == 64) return launch_halo_t<BN, 64, true>(st, ntiles, h, B, e, err);
        if (CS == 32) return launch_halo_t<BN, 32, true>(st, ntiles, h, B, e, err);
    } else {
        if (CS == 64) return launch_halo_t<BN, 64, false>(st, ntiles, h, B, e, err);
        if (CS == 32) return launch_halo_t<BN, 32, false>(st, ntiles, h, B, e, err);
        if (CS == 16) return launch_halo_t<BN, 16, false>(st, ntiles, h, B, e, err);
    }
    return fail(WEC_ERR_INVALID, "net: unsupported channels per stage");
}

// A convolution of the given HaloMode whose output grid is the level's: input
// channels [0, c0) from in0 and [c0, c0 + c1) from in1 (concatenation; c1 = 0:
// one tensor), ncols output channels, halo-ordered weights B of tile width BN.
int conv_halo(wec_net *N, cudaStream_t st, int tag, int mode, int batch, int level, const bf16 *in0, int c0,
              const bf16 *in1, int c1, const bf16 *B, int BN, int ncols, const Epi &e)
{
    Halo h{};
    h.in0 = in0;
    h.in1 = in1 ? in1 : in0;
    h.c0 = c0;
    h.c1 = in1 ? c1 : 0;
    h.N = batch;
    h.H = level_h(N, level);
    h.W = level_w(N, level);
    h.Hi = mode == H_UP3 ? h.H / 2 : (mode == H_DOWN2 ? 2 * h.H : h.H);
    h.Wi = mode == H_UP3 ? h.W / 2 : (mode == H_DOWN2 ? 2 * h.W : h.W);
    h.xtiles = ((mode == H_UP3 ? h.Wi : h.W) + kBM - 1) / kBM;  // the up mode tiles its input row
    h.mode = mode;
    const int CS = halo_cs(c0), tv = mode == H_DOWN2 ? 2 : 3;
    h.nst = (h.c0 + h.c1) / CS * tv;
    h.ncols = ncols;
    const long long ntiles = (long long)batch * h.H * h.xtiles * (ncols / BN);
    const double M = (double)batch * h.H * h.W;
    WEC_PROF("net_conv", tag, 2.0 * M * ((double)(h.c0 + h.c1) + ncols) + 2.0 * tv * tv * (h.c0 + h.c1) * ncols, st);
    switch (BN) {
    case 128: return launch_halo_cs<128>(CS, mode == H_DOWN2, st, ntiles, h, B, e, N->err);
    case 64: return launch_halo_cs<64>(CS, mode == H_DOWN2, st, ntiles, h, B, e, N->err);
    default: return launch_halo_cs<32>(CS, mode == H_DOWN2, st, ntiles, h, B, e, N->err);
    }
}

int wgrad_splits(long long M, int L, int *cps)
{
    const int co = kLayers[L].co, BN = co % 64 == 0 ? 64 : 32;
    const int tiles = round_up(fwd_K(L), kBM) / kBM * (co / BN);
    const int nchunks = (int)((M + kBK - 1) / kBK);
    int splits = std::max(1, std::min((kWgradTarget + tiles - 1) / tiles, nchunks));
    *cps = (nchunks + splits - 1) / splits;
    return (nchunks + *cps - 1) / *cps;
}

// grad of layer L's weights and bias from its output gradient G.
int wgrad(wec_net *N, int L, int batch, const bf16 *G)
{
    const LayerDef &d = kLayers[L];
    const Gat g = fwd_gather(N, L, batch);
    const long long M = (long long)g.N * g.H * g.W;
    const int Kw = round_up(g.K, kBM), BN = d.co % 64 == 0 ? 64 : 32;
    int cps = 0;
    const int splits = wgrad_splits(M, L, &cps);
    cudaStream_t st = N->st;
    {
        WEC_PROF("net_wgrad", -1, 2.0 * M * ((double)(g.c0 + g.c1) * taps(d.kind) + d.co), st);
        dim3 grid((unsigned)(Kw / kBM), (unsigned)(d.co / BN), (unsigned)splits);
        if (BN == 64)
            WEC_CK(launch_k(k_wgrad<64>, grid, kGT, 0, st, g, G, d.co, cps, Kw, N->part));
        else
            WEC_CK(launch_k(k_wgrad<32>, grid, kGT, 0, st, g, G, d.co, cps, Kw, N->part));
    }
    float *gw = N->grad + N->flat[L];
    const long long nw = (long long)weight_count(L);
    {
        WEC_PROF("net_wgrad_reduce", -1, 4.0 * nw * (splits + 1), st);
        WEC_CK(launch_k(k_wgrad_reduce, nblk(nw, kT), kT, 0, st, (const float *)N->part, splits, Kw, d.co,
                        cin_pad(d.ci), d.ci, taps(d.kind), gw));
    }
    const int rows = g.N * g.H;
    const int nb = std::min(kCsumBlocks, rows);
    const int rpb = (rows + nb - 1) / nb;
    {
        WEC_PROF("net_bias_grad", -1, 2.0 * M * d.co, st);
        WEC_CK(launch_k(k_colsum, nb, kT, 0, st, G, rows, g.W, d.co, rpb, N->cpart));
    }
    {
        WEC_PROF("net_bias_grad", -1, 4.0 * nb * d.co, st);
        WEC_CK(launch_k(k_colsum_final, nblk(d.co, kT), kT, 0, st, (const float *)N->cpart, nb, d.co, gw + nw));
    }
    return WEC_OK;
}

// Input gradient of a 3x3 layer (conv or up): the 3x3 convolution of G (its
// output gradient, level grid) with the flipped, transposed weights.
int dx_conv(wec_net *N, int L, int batch, const bf16 *G, const Epi &e)
{
    const LayerDef &d = kLayers[L];
    return conv_halo(N, N->st, 100 + L, H_CONV3, batch, d.level, G, d.co, nullptr, 0, N->wmat + N->hb[L], N->bnb[L],
                     d.ci, e);
}

int pack_weights(wec_net *N)
{
    for (int L = 0; L < kHead; ++L) {
        const LayerDef &d = kLayers[L];
        if (d.kind == L_DOWN2) {
            const long long n = (long long)weight_count(L);
            WEC_PROF("net_pack", -1, 6.0 * n, N->st);
            WEC_CK(launch_k(k_pack_down, nblk(n, kT), kT, 0, N->st, (const float *)(N->theta + N->flat[L]), n,
                            N->wmat + N->wb[L]));
        }
        for (int bwd = 0; bwd < 2; ++bwd) {
            if (!(bwd ? halo_bwd(L) : halo_fwd(L))) continue;
            const int kin = halo_kin(L, bwd), ncols = bwd ? d.ci : d.co, BN = bwd ? N->bnb[L] : N->bnf[L];
            const bool concat = L == cat(0) || L == cat(1) || L == cat(2);
            const int cs = halo_cs(bwd ? d.co : (concat ? d.ci / 2 : kin));
            const int tv = (!bwd && d.kind == L_DOWN2) ? 2 : 3;
            const long long nh = (long long)tv * tv * kin * ncols;
            WEC_PROF("net_pack", -1, 4.0 * weight_count(L) + 2.0 * nh, N->st);
            WEC_CK(launch_k(k_pack_halo, nblk(nh, kT), kT, 0, N->st, (const float *)(N->theta + N->flat[L]), d.ci,
                            d.co, kin, ncols, BN, cs, tv, tv, bwd, N->wmat + (bwd ? N->hb[L] : N->hf[L])));
        }
    }
    N->wdirty = false;
    return WEC_OK;
}

// Forward pass of batch images x (FP32 [batch][H][W][2]) into out; with a
// target, also the head's gradient, loss partials and G of dec0 (in gA[0]).
int forward(wec_net *N, int batch, const float *x, float *out, const float *target)
{
    cudaStream_t st = N->st;
    if (N->wdirty)
        if (int e = pack_weights(N)) return e;
    const long long M = (long long)batch * N->H * N->W;
    {
        WEC_PROF("net_input", -1, 8.0 * M + 16.0 * M, st);
        WEC_CK(launch_k(k_input, nblk(M, kT), kT, 0, st, x, M, N->W, N->xin));
    }
    for (int L = 0; L < kHead; ++L) {
        const LayerDef &d = kLayers[L];
        Epi e{};
        e.kind = E_FWD;
        e.bias = N->theta + N->flat[L] + weight_count(L);
        e.out0 = N->act[L];
        e.ld0 = d.co;
        const Gat g = fwd_gather(N, L, batch);
        if (int r = conv_halo(N, st, L, halo_mode(d.kind), batch, d.level, g.in0, g.c0, g.in1, g.c1,
                              N->wmat + N->hf[L], N->bnf[L], d.co, e))
            return r;
    }
    const int nb = nblk(M, kT);
    {
        WEC_PROF("net_head", -1, 64.0 * M + 8.0 * M, st);
        WEC_CK(launch_k(k_head, nb, kT, 0, st, (const bf16 *)N->act[dec(0)], (const float *)(N->theta + N->flat[kHead]),
                        M, N->W, out, target, (float)(1.0 / (double)M), N->gA[0], N->cpart));
    }
    if (target) {
        WEC_PROF("net_head", -1, 4.0 * kHeadVals * nb, st);
        WEC_CK(launch_k(k_head_final, 1, 64, 0, st, (const float *)N->cpart, nb, N->grad + N->flat[kHead], N->loss,
                        1.0 / (double)M));
    }
    return WEC_OK;
}

int backward(wec_net *N, int batch)
{
    cudaStream_t st = N->st;
    for (int l = 0; l < 3; ++l) {  // decoder, last level first; G of dec(l) is in gA[l]
        const int C = chans(l);
        if (int r = wgrad(N, dec(l), batch, N->gA[l])) return r;
        Epi e{};
        e.kind = E_DX;
        e.out0 = N->gB[l];
        e.mask0 = N->act[cat(l)];
        e.ld0 = C;
        e.nsplit = C;
        if (int r = dx_conv(N, dec(l), batch, N->gA[l], e)) return r;
        if (int r = wgrad(N, cat(l), batch, N->gB[l])) return r;
        e.out0 = N->gA[l];
        e.mask0 = N->act[up(l)];
        e.out1 = N->skip[l];
        e.ld1 = C;
        if (int r = dx_conv(N, cat(l), batch, N->gB[l], e)) return r;
        if (int r = wgrad(N, up(l), batch, N->gA[l])) return r;
        Epi f{};
        f.kind = E_F32;
        f.outf = N->tmpf;
        f.ld0 = 2 * C;
        if (int r = dx_conv(N, up(l), batch, N->gA[l], f)) return r;
        const int h = level_h(N, l + 1), w = level_w(N, l + 1);
        const long long n = (long long)batch * h * w * 2 * C;
        WEC_PROF("net_up_pool", -1, 16.0 * n + 4.0 * n, st);
        WEC_CK(launch_k(k_up_pool, nblk(n, kT), kT, 0, st, (const float *)N->tmpf,
                        (const bf16 *)(l == 2 ? N->act[enc_b(3)] : N->act[dec(l + 1)]), batch, h, w, 2 * C,
                        N->gA[l + 1]));
    }
    for (int l = 3; l >= 0; --l) {  // encoder; G of down(l)'s output is in gA[l + 1]
        const int C = chans(l);
        if (l < 3) {
            if (int r = wgrad(N, down(l), batch, N->gA[l + 1])) return r;
            Gat g{};
            g.in0 = N->gA[l + 1];
            g.c0 = 2 * C;
            g.lcin = ilog2(2 * C);
            g.kind = G_DIRECT;
            g.N = batch;
            g.H = g.Hi = level_h(N, l + 1);
            g.W = g.Wi = level_w(N, l + 1);
            g.K = 2 * C;
            Epi e{};
            e.kind = E_DOWNDX;
            e.out0 = N->gA[l];
            e.mask0 = N->act[enc_b(l)];
            e.ld0 = C;
            e.add = N->skip[l];
            if (int r = gemm(N, st, 100 + down(l), g, N->wmat + N->wb[down(l)], 2 * C, (size_t)2 * C * C, C, 4, e))
                return r;
        }
        if (int r = wgrad(N, enc_b(l), batch, N->gA[l])) return r;
        Epi e{};
        e.kind = E_DX;
        e.out0 = N->gB[l];
        e.mask0 = N->act[enc_a(l)];
        e.ld0 = C;
        e.nsplit = C;
        if (int r = dx_conv(N, enc_b(l), batch, N->gA[l], e)) return r;
        if (int r = wgrad(N, enc_a(l), batch, N->gB[l])) return r;
        if (l > 0) {
            e.out0 = N->gA[l];
            e.mask0 = N->act[down(l - 1)];
            if (int r = dx_conv(N, enc_a(l), batch, N->gB[l], e)) return r;
        }
    }
    return WEC_OK;
}

int net_alloc(wec_net *N, void **p, size_t bytes)
{
    cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 256));
    if (e != cudaSuccess) return cuda_fail(e, "net: device allocation");
    N->allocs.push_back(*p);
    return WEC_OK;
}

void net_free(wec_net *N)
{
    if (!N) return;
    if (N->st) cudaStreamSynchronize(N->st);
    for (void *p : N->allocs) cudaFree(p);
    if (N->lossh) cudaFreeHost(N->lossh);
    delete N;
}

}  // namespace

size_t net_param_count()
{
    size_t n = 0;
    for (int L = 0; L < kNumLayers; ++L) n += weight_count(L) + kLayers[L].co;
    return n;
}

int net_sync_weights(wec_net *N)
{
    if (!N->wdirty) return WEC_OK;
    if (int r = pack_weights(N)) return r;
    WEC_CK(cudaStreamSynchronize(N->st));
    return WEC_OK;
}

// Enqueue the net's guess for the tank's increment phi (step front, after the
// pressure problem is built).
int net_enqueue_guess(wec_tank *T, cudaStream_t st)
{
    wec_net *N = T->net;
    if (N->wdirty) return fail(WEC_ERR_INVALID, "net guess: BF16 weights not packed");
    const int nx = T->P.nx, ny = T->P.ny, nc = nx * ny;
    const double *bu = T->solver.L64[0].bu, *bv = T->solver.L64[0].bv;
    cudaStream_t keep = N->st;
    N->st = st;
    {
        WEC_PROF("net_features", -1, 8.0 * nc, st);
        WEC_CK(launch_k(k_feat_bsum, kRedBlocks, kT, 0, st, (const double *)T->rhs, nc, N->dpart));
    }
    {
        WEC_PROF("net_features", -1, 8.0 * nc * 4 + 8.0 * nc, st);
        WEC_CK(launch_k(k_features, nblk(nc, kT), kT, 0, st, nx, ny, (const double *)T->rhs, bu, bv,
                        (const double *)T->inp, T->P.rho_w, (const double *)N->dpart, kRedBlocks,
                        (const double *)nullptr, N->xb, (float *)nullptr));
    }
    int r = forward(N, 1, N->xb, N->out, nullptr);
    N->st = keep;
    if (r) return r;
    {
        WEC_PROF("net_guess", -1, 8.0 * nc * 4 + 4.0 * nc, st);
        WEC_CK(launch_k(k_guess, nblk(nc, kT), kT, 0, st, nx, ny, (const double *)T->rhs, bu, bv,
                        (const double *)N->dpart, kRedBlocks, (const float *)N->out, T->phi));
    }
    {
        WEC_PROF("net_guess", -1, 8.0 * nc * 5, st);
        WEC_CK(launch_k(k_guess_resid, kRedBlocks, kT, 0, st, nx, ny, (const double *)T->rhs, bu, bv,
                        (const double *)T->phi, N->dpart + kRedBlocks));
    }
    {
        WEC_PROF("net_guess", -1, 8.0 * nc, st);
        WEC_CK(launch_k(k_guess_select, nblk(nc, kT), kT, 0, st, nc, (const double *)N->dpart,
                        (const double *)(N->dpart + kRedBlocks), kRedBlocks, T->phi, T->net_stats));
    }
    return WEC_OK;
}

}  // namespace wec

using namespace wec;

extern "C" {

size_t wec_net_param_count(void) { return net_param_count(); }

int wec_net_create(int H, int W, int max_batch, void *cuda_stream, wec_net **out)
{
    if (!out) return fail(WEC_ERR_INVALID, "net_create: out is NULL");
    *out = nullptr;
    if (H < 8 || W < 8 || H % 8 || W % 8 || max_batch < 1)
        return fail(WEC_ERR_INVALID, "net_create: H, W must be multiples of 8 (>= 8) and max_batch >= 1");
    if ((long long)H * W * max_batch > (1LL << 26))
        return fail(WEC_ERR_INVALID, "net_create: max_batch * H * W above 2^26 pixels");
    wec_net *N = new (std::nothrow) wec_net();
    if (!N) return fail(WEC_ERR_NOMEM, "net_create: host allocation failed");
    N->H = H;
    N->W = W;
    N->maxb = max_batch;
    N->st = (cudaStream_t)cuda_stream;
    N->nparam = net_param_count();
    size_t nw = 0, off = 0;
    for (int L = 0; L < kNumLayers; ++L) {
        N->flat[L] = off;
        off += weight_count(L) + kLayers[L].co;
        if (L == kHead) break;
        const LayerDef &d = kLayers[L];
        if (d.kind == L_DOWN2) {
            N->wb[L] = nw;
            nw = round_up_z(nw + weight_count(L), 64);
        }
        if (halo_fwd(L)) {
            N->bnf[L] = halo_bn(N, d.level, d.co, d.kind == L_UP3);
            N->hf[L] = nw;
            nw = round_up_z(nw + (size_t)taps(d.kind) * halo_kin(L, false) * d.co, 64);
        }
        if (halo_bwd(L)) {
            N->bnb[L] = halo_bn(N, d.level, d.ci);
            N->hb[L] = nw;
            nw = round_up_z(nw + 9 * (size_t)halo_kin(L, true) * d.ci, 64);
        }
    }
    const size_t P0 = (size_t)max_batch * H * W;
    auto pix = [&](int l) { return P0 >> (2 * l); };
    size_t part_n = 0;
    for (int L = 0; L < kHead; ++L) {
        int cps = 0;
        const int s = wgrad_splits((long long)pix(kLayers[L].level), L, &cps);
        part_n = std::max(part_n, (size_t)s * round_up(fwd_K(L), kBM) * kLayers[L].co);
    }
    int r = WEC_OK;
    auto A = [&](void **p, size_t bytes) {
        if (!r) r = net_alloc(N, p, bytes);
    };
    A((void **)&N->theta, 4 * N->nparam);
    A((void **)&N->grad, 4 * N->nparam);
    A((void **)&N->am, 4 * N->nparam);
    A((void **)&N->av, 4 * N->nparam);
    A((void **)&N->wmat, 2 * nw);
    A((void **)&N->xin, 2 * P0 * kInPad);
    for (int L = 0; L < kHead; ++L) A((void **)&N->act[L], 2 * pix(kLayers[L].level) * kLayers[L].co);
    A((void **)&N->out, 4 * P0);
    for (int l = 0; l < 4; ++l) {
        A((void **)&N->gA[l], 2 * pix(l) * chans(l));
        A((void **)&N->gB[l], 2 * pix(l) * chans(l));
        if (l < 3) A((void **)&N->skip[l], 2 * pix(l) * chans(l));
    }
    A((void **)&N->tmpf, 4 * P0 * 64);
    A((void **)&N->part, 4 * part_n);
    A((void **)&N->cpart, 4 * (size_t)std::max(kCsumBlocks * 256, nblk((long long)P0, kT) * kHeadVals));
    A((void **)&N->xb, 4 * P0 * kInCh);
    A((void **)&N->tb, 4 * P0);
    A((void **)&N->loss, 8);
    A((void **)&N->dpart, 8 * 2 * kRedBlocks);
    A((void **)&N->err, sizeof(int));
    N->part_n = part_n;
    if (!r) {
        cudaError_t ce = cudaMallocHost((void **)&N->lossh, 8);
        if (ce != cudaSuccess) r = cuda_fail(ce, "net_create: pinned allocation");
    }
    if (!r) {
        cudaError_t ce = cudaMemsetAsync(N->theta, 0, 4 * N->nparam, N->st);
        if (ce == cudaSuccess) ce = cudaMemsetAsync(N->grad, 0, 4 * N->nparam, N->st);
        if (ce == cudaSuccess) ce = cudaMemsetAsync(N->am, 0, 4 * N->nparam, N->st);
        if (ce == cudaSuccess) ce = cudaMemsetAsync(N->av, 0, 4 * N->nparam, N->st);
        if (ce == cudaSuccess) ce = cudaMemsetAsync(N->err, 0, sizeof(int), N->st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(N->st);
        if (ce != cudaSuccess) r = cuda_fail(ce, "net_create: initialisation");
    }
    if (r) {
        net_free(N);
        return r;
    }
    *out = N;
    return WEC_OK;
}

void wec_net_destroy(wec_net *N) { net_free(N); }

int wec_net_set_params(wec_net *N, const float *host, size_t n)
{
    if (!N || !host) return fail(WEC_ERR_INVALID, "net_set_params: NULL argument");
    if (n != N->nparam) return fail(WEC_ERR_INVALID, "net_set_params: n must equal wec_net_param_count()");
    for (size_t k = 0; k < n; ++k)
        if (!std::isfinite(host[k])) return fail(WEC_ERR_INVALID, "net_set_params: non-finite parameter");
    WEC_CK(cudaMemcpyAsync(N->theta, host, 4 * n, cudaMemcpyHostToDevice, N->st));
    WEC_CK(cudaMemsetAsync(N->am, 0, 4 * n, N->st));
    WEC_CK(cudaMemsetAsync(N->av, 0, 4 * n, N->st));
    WEC_CK(cudaStreamSynchronize(N->st));
    N->adam_t = 0;
    N->wdirty = true;
    return WEC_OK;
}

// After a synchronising call: a tensor-core pipeline wait that expired is an error.
static int check_pipeline(wec_net *N, const char *what)
{
    int h = 0;
    WEC_CK(cudaMemcpy(&h, N->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (!h) return WEC_OK;
    WEC_CK(cudaMemset(N->err, 0, sizeof(int)));
    return fail(WEC_ERR_CUDA, std::string(what) + ": a tensor-core pipeline wait expired");
}

static int copy_out(const wec_net *N, const float *src, float *host, size_t n, const char *what)
{
    if (!N || !host) return fail(WEC_ERR_INVALID, std::string(what) + ": NULL argument");
    if (n != N->nparam) return fail(WEC_ERR_INVALID, std::string(what) + ": n must equal wec_net_param_count()");
    WEC_CK(cudaMemcpyAsync(host, src, 4 * n, cudaMemcpyDeviceToHost, N->st));
    WEC_CK(cudaStreamSynchronize(N->st));
    return WEC_OK;
}

int wec_net_get_params(const wec_net *N, float *host, size_t n)
{
    return copy_out(N, N ? N->theta : nullptr, host, n, "net_get_params");
}

int wec_net_get_grads(const wec_net *N, float *host, size_t n)
{
    return copy_out(N, N ? N->grad : nullptr, host, n, "net_get_grads");
}

int wec_net_get_activation(const wec_net *N, int layer, int batch, unsigned short *host, size_t n)
{
    if (!N || !host) return fail(WEC_ERR_INVALID, "net_get_activation: NULL argument");
    if (layer < 0 || layer >= kHead || batch < 1 || batch > N->maxb)
        return fail(WEC_ERR_INVALID, "net_get_activation: layer outside [0, 19] or batch outside [1, max_batch]");
    const LayerDef &d = kLayers[layer];
    const size_t want = (size_t)batch * level_h(N, d.level) * level_w(N, d.level) * d.co;
    if (n != want) return fail(WEC_ERR_INVALID, "net_get_activation: n does not match the layer's tensor");
    WEC_CK(cudaMemcpyAsync(host, N->act[layer], 2 * n, cudaMemcpyDeviceToHost, N->st));
    WEC_CK(cudaStreamSynchronize(N->st));
    return WEC_OK;
}

int wec_net_forward(wec_net *N, int batch, const float *x, float *out)
{
    if (!N || !x || !out) return fail(WEC_ERR_INVALID, "net_forward: NULL argument");
    if (batch < 1 || batch > N->maxb) return fail(WEC_ERR_INVALID, "net_forward: batch outside [1, max_batch]");
    if (int r = forward(N, batch, x, out, nullptr)) return r;
    WEC_CK(cudaStreamSynchronize(N->st));
    return check_pipeline(N, "net_forward");
}

int wec_net_loss_grad(wec_net *N, int batch, const float *x, const float *target, double *loss)
{
    if (!N || !x || !target || !loss) return fail(WEC_ERR_INVALID, "net_loss_grad: NULL argument");
    if (batch < 1 || batch > N->maxb) return fail(WEC_ERR_INVALID, "net_loss_grad: batch outside [1, max_batch]");
    if (int r = forward(N, batch, x, N->out, target)) return r;
    if (int r = backward(N, batch)) return r;
    WEC_CK(cudaMemcpyAsync(N->lossh, N->loss, 8, cudaMemcpyDeviceToHost, N->st));
    WEC_CK(cudaStreamSynchronize(N->st));
    if (int r = check_pipeline(N, "net_loss_grad")) return r;
    *loss = *N->lossh;
    return std::isfinite(*loss) ? WEC_OK : fail(WEC_ERR_NONFINITE, "net_loss_grad: non-finite loss");
}

int wec_net_adam(wec_net *N, float lr)
{
    if (!N) return fail(WEC_ERR_INVALID, "net_adam: NULL net");
    if (!(lr > 0.0f) || !std::isfinite(lr)) return fail(WEC_ERR_INVALID, "net_adam: lr must be finite and > 0");
    N->adam_t += 1;
    const float b1t = (float)(1.0 - std::pow(0.9, (double)N->adam_t));
    const float b2t = (float)(1.0 - std::pow(0.999, (double)N->adam_t));
    {
        WEC_PROF("net_adam", -1, 4.0 * 7 * N->nparam, N->st);
        WEC_CK(launch_k(k_adam, nblk((long long)N->nparam, kT), kT, 0, N->st, N->theta, (const float *)N->grad, N->am,
                        N->av, (long long)N->nparam, lr, b1t, b2t));
    }
    N->wdirty = true;
    return WEC_OK;
}

int wec_net_train_step(wec_net *N, const float *xs, const float *ts, const int *idx, int batch, float lr,
                       double *loss)
{
    if (!N || !xs || !ts || !idx || !loss) return fail(WEC_ERR_INVALID, "net_train_step: NULL argument");
    if (batch < 1 || batch > N->maxb) return fail(WEC_ERR_INVALID, "net_train_step: batch outside [1, max_batch]");
    const size_t px = (size_t)N->H * N->W;
    for (int b = 0; b < batch; ++b) {
        if (idx[b] < 0) return fail(WEC_ERR_INVALID, "net_train_step: negative sample index");
        WEC_CK(cudaMemcpyAsync(N->xb + b * px * kInCh, xs + (size_t)idx[b] * px * kInCh, 4 * px * kInCh,
                               cudaMemcpyDeviceToDevice, N->st));
        WEC_CK(cudaMemcpyAsync(N->tb + b * px, ts + (size_t)idx[b] * px, 4 * px, cudaMemcpyDeviceToDevice, N->st));
    }
    if (int r = wec_net_loss_grad(N, batch, N->xb, N->tb, loss)) return r;
    return wec_net_adam(N, lr);
}

int wec_net_sample(wec_tank *T, float *x, float *t)
{
    if (!T || !x || !t) return fail(WEC_ERR_INVALID, "net_sample: NULL argument");
    if (!T->stepped) return fail(WEC_ERR_INVALID, "net_sample: the tank has not stepped yet");
    const int nx = T->P.nx, ny = T->P.ny, nc = nx * ny;
    cudaStream_t st = T->gst;
    {
        WEC_PROF("net_features", -1, 8.0 * nc, st);
        WEC_CK(launch_k(k_feat_bsum, kRedBlocks, kT, 0, st, (const double *)T->rhs, nc, T->part));
    }
    {
        WEC_PROF("net_features", -1, 8.0 * nc * 6 + 12.0 * nc, st);
        WEC_CK(launch_k(k_features, nblk(nc, kT), kT, 0, st, nx, ny, (const double *)T->rhs,
                        (const double *)T->solver.L64[0].bu, (const double *)T->solver.L64[0].bv,
                        (const double *)T->inp, T->P.rho_w, (const double *)T->part, kRedBlocks,
                        (const double *)T->phi, x, t));
    }
    WEC_CK(cudaStreamSynchronize(st));
    return WEC_OK;
}

int wec_tank_set_net(wec_tank *T, wec_net *N)
{
    if (!T) return fail(WEC_ERR_INVALID, "tank_set_net: NULL tank");
    if (N && (N->H != T->P.ny || N->W != T->P.nx))
        return fail(WEC_ERR_INVALID, "tank_set_net: the net's H x W must be the tank's ny x nx");
    if (!T->inp_owned) return fail(WEC_ERR_INVALID, "tank_set_net: tanks of a batch take no net");
    if (N)
        if (int r = net_sync_weights(N)) return r;
    if (!T->net_stats) {
        WEC_CK(cudaMalloc(&T->net_stats, 2 * sizeof(long long)));
        WEC_CK(cudaMemsetAsync(T->net_stats, 0, 2 * sizeof(long long), T->gst));
        WEC_CK(cudaStreamSynchronize(T->gst));
    }
    WEC_CK(cudaStreamSynchronize(T->gst));
    if (T->exec) cudaGraphExecDestroy(T->exec);
    if (T->graph) cudaGraphDestroy(T->graph);
    T->exec = nullptr;
    T->graph = nullptr;
    T->net = N;
    return WEC_OK;
}

int wec_tank_net_stats(const wec_tank *T, long long *tried, long long *kept)
{
    if (!T || !tried || !kept) return fail(WEC_ERR_INVALID, "tank_net_stats: NULL argument");
    long long h[2] = {0, 0};
    if (T->net_stats) {
        WEC_CK(cudaMemcpyAsync(h, T->net_stats, sizeof(h), cudaMemcpyDeviceToHost, T->gst));
        WEC_CK(cudaStreamSynchronize(T->gst));
    }
    *tried = h[0];
    *kept = h[1];
    return WEC_OK;
}

}  // extern "C"
