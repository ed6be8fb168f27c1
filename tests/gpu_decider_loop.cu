// Replica of the Ising decider's 32-site loop, timed alone on one warp per block
// (test infrastructure: it measures the chain-latency bound that the benchmark
// reports; it is not part of the library).
//
// It runs the loop of the kernel's Ising stream decider: byte-parallel constants of
// four sites (one prmt per constant), the bin and its change selected by the previous
// decision, the two candidate thresholds of the next site loaded before the current
// site is decided, then select -> compare.  Output: cycles per site (clock64).
// Thresholds are random; the rows of the NB_EDGE lowest and highest bins are 0 (never
// accept), so every bin, including the speculative ones two moves ahead, stays inside
// the table.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
constexpr int NBINS = 4097, NB_EDGE = 8;

__device__ __forceinline__ uint32_t lds_u32(uint32_t a) { uint32_t v; asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a)); return v; }

struct Word { uint32_t lo, hi, qw; };
__device__ __forceinline__ uint32_t ubyte(uint32_t x, int k)
{
    uint32_t d;
    asm("prmt.b32 %0, %1, 0, %2;" : "=r"(d) : "r"(x), "r"(0x4440u | (uint32_t)k));
    return d;
}
__device__ __forceinline__ uint32_t sbyte(uint32_t x, int k)
{
    uint32_t d;
    asm("prmt.b32 %0, %1, 0, %2;" : "=r"(d) : "r"(x), "r"((uint32_t)k | (8u | (uint32_t)k) * 0x1110u));
    return d;
}
struct Quad { uint32_t K0, K1, D0, D1; };
__device__ __forceinline__ uint32_t spread4(uint32_t x, int g, int s)
{
    return (((x >> (4 * g)) & 0xFu) * (0x00204081u << s)) & (0x01010101u << s);
}
__device__ __forceinline__ Quad quad(const Word &x, int g)
{
    const uint32_t pre4 = spread4(x.lo, g, 2) + spread4(x.hi, g, 3), q4 = spread4(x.qw, g, 2);
    Quad r;
    r.K0 = pre4 + q4;
    r.K1 = pre4 + 0x04040404u - q4;
    r.D0 = (0xA8A8A8A8u - 5u * r.K0) ^ 0x80808080u;
    r.D1 = (0xA8A8A8A8u - 5u * r.K1) ^ 0x80808080u;
    return r;
}
__device__ __forceinline__ uint32_t lcg(uint32_t &s) { s = s * 1664525u + 1013904223u; return s; }

__global__ void __launch_bounds__(32) k(const uint32_t *gtab, int n_words, uint32_t *out, long long *cyc)
{
    extern __shared__ uint32_t sm[];
    uint32_t *tab = sm;                         // NBINS*5
    uint4 *drw = reinterpret_cast<uint4 *>(sm + ((NBINS * 5 + 3) & ~3));  // [8][32] draws of a word
    for (int i = threadIdx.x; i < NBINS * 5; i += 32) tab[i] = gtab[i];
    const int lane = threadIdx.x;
    const int cl = lane;
    uint32_t s = 12345u + cl * 7919u;
    for (int i = 0; i < 8; ++i) drw[i * 32 + lane] = make_uint4(lcg(s), lcg(s), lcg(s), lcg(s));
    __syncwarp();
    const uint32_t tab_s = (uint32_t)__cvta_generic_to_shared(tab);
    uint32_t P0 = 20u * (NBINS / 2 + (cl & 7)), P1 = P0;
    bool ap = false;
    uint32_t Racc = 0;
    long long t0 = clock64();
    Word cur{lcg(s), lcg(s), lcg(s)};
    {
        // P0 / P1 absolute table addresses of the current site's bin
        P0 += tab_s;
        P1 += tab_s;
        Quad q0 = quad(cur, 0);
        uint32_t A0 = lds_u32(P0 + ubyte(q0.K0, 0)), A1 = lds_u32(P1 + ubyte(q0.K1, 0));
        for (int wi = 0; wi < n_words; ++wi) {
            Word nx{cur.lo * 3u + lcg(s), cur.hi ^ lcg(s), cur.qw + lcg(s)};
            uint4 blk = drw[lane], blk_next = drw[32 + lane];
            uint32_t Rw = 0;
            Quad q1 = quad(cur, 1);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int kk = j & 3;
                if (kk == 0 && j > 0) {
                    blk = blk_next;
                    if (j < 28) blk_next = drw[((j >> 2) + 1) * 32 + lane];
                    q0 = q1;
                    q1 = j < 28 ? quad(cur, (j >> 2) + 1) : quad(nx, 0);
                }
                const uint32_t u = min(kk == 0 ? blk.x : kk == 1 ? blk.y : kk == 2 ? blk.z : blk.w, 0xFFFFFFFEu);
                const uint32_t Pc = ap ? P1 : P0;
                const uint32_t DD = ap ? sbyte(q0.D1, kk) : sbyte(q0.D0, kk);
                const uint32_t nP1 = Pc + DD;
                const uint32_t K0n = kk == 3 ? ubyte(q1.K0, 0) : ubyte(q0.K0, kk + 1);
                const uint32_t K1n = kk == 3 ? ubyte(q1.K1, 0) : ubyte(q0.K1, kk + 1);
                const uint32_t A0n = lds_u32(Pc + K0n), A1n = lds_u32(nP1 + K1n);
                const uint32_t A = ap ? A1 : A0;
                const bool acc = u < A;
                A0 = A0n;
                A1 = A1n;
                P0 = Pc;
                P1 = nP1;
                Rw ^= acc ? (1u << j) : 0u;
                ap = acc;
            }
            q0 = q1;
            Racc += Rw;
            cur = nx;
        }
    }
    long long t1 = clock64();
    out[blockIdx.x * 32 + lane] = Racc ^ P0 ^ P1;
    if (lane == 0) cyc[blockIdx.x] = t1 - t0;
}


int main()
{
    const int n_words = 2048, blocks = 32;
    uint32_t *h = new uint32_t[NBINS * 5];
    uint32_t s = 1;
    for (int b = 0; b < NBINS; ++b)
        for (int c = 0; c < 5; ++c) {
            s = s * 1664525u + 1013904223u;
            h[b * 5 + c] = (b < NB_EDGE || b >= NBINS - NB_EDGE) ? 0u : s;
        }
    uint32_t *gtab, *out; long long *cyc;
    cudaMalloc(&gtab, NBINS * 5 * 4); cudaMalloc(&out, blocks * 32 * 4); cudaMalloc(&cyc, blocks * 8);
    cudaMemcpy(gtab, h, NBINS * 5 * 4, cudaMemcpyHostToDevice);
    const size_t smem = ((NBINS * 5 + 3) & ~3) * 4 + 8 * 32 * 16;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<blocks, 32, smem>>>(gtab, n_words, out, cyc);
    if (cudaDeviceSynchronize() != cudaSuccess) { printf("error\n"); return 1; }
    long long c[blocks]; cudaMemcpy(c, cyc, sizeof c, cudaMemcpyDeviceToHost);
    double m = 0; for (int i = 0; i < blocks; ++i) m += c[i];
    printf("decider loop: %.1f cycles/site\n", m / blocks / (n_words * 32.0));
    return 0;
}
