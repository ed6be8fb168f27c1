// Replica of the Ising decider's 32-site loop, timed alone on one warp per block
// (test infrastructure: it measures the chain-latency bound that the benchmark
// reports; it is not part of the library).
//
// Modes (cycles per site, clock64):
//   0  the loop as in the kernel: per-site constants from bit-sliced neighbour counts,
//      two speculative table loads (offsets resolved by the previous decision),
//      select -> compare
//   1  speculation two sites deep (four table loads per site)
//   2  mode 0 with thresholds computed by ALU instead of loaded
//   3  ALU thresholds and fixed per-site constants
//   4  table loads and fixed per-site constants
//   5  the accept chain alone (select -> compare)
//   6-9  modes 4 and 0 with the compare ordered after the loads (a volatile move, or
//        loads and compare in one asm block)
//   10   the loop as in the kernel now: byte-parallel constants of four sites, one
//        prmt per constant, the bin and its change selected by the previous decision
//   11, 12  mode 10 with 16 / 8 distinct chains per warp (lanes l and l + 16, or
//        l mod 8, run the same chain: same addresses, so fewer bank conflicts)
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

template <int MODE>
__global__ void __launch_bounds__(32) k(const uint32_t *gtab, int n_words, uint32_t *out, long long *cyc)
{
    extern __shared__ uint32_t sm[];
    uint32_t *tab = sm;                         // NBINS*5
    uint4 *drw = reinterpret_cast<uint4 *>(sm + ((NBINS * 5 + 3) & ~3));  // [8][32] draws of a word
    for (int i = threadIdx.x; i < NBINS * 5; i += 32) tab[i] = gtab[i];
    const int lane = threadIdx.x;
    // distinct chains per warp: 32, or 16 / 8 with the other lanes repeating them
    const int cl = MODE == 11 ? (lane & 15) : MODE == 12 ? (lane & 7) : lane;
    uint32_t s = 12345u + cl * 7919u;
    for (int i = 0; i < 8; ++i) drw[i * 32 + lane] = make_uint4(lcg(s), lcg(s), lcg(s), lcg(s));
    __syncwarp();
    const uint32_t tab_s = (uint32_t)__cvta_generic_to_shared(tab);
    uint32_t P0 = 20u * (NBINS / 2 + (cl & 7)), P1 = P0;
    bool ap = false;
    uint32_t Racc = 0;
    long long t0 = clock64();
    Word cur{lcg(s), lcg(s), lcg(s)};
    auto consts = [&](const Word &x, int j, uint32_t &K0, uint32_t &K1, uint32_t &D0, uint32_t &D1) {
        const uint32_t pre = ((x.lo >> j) & 1u) + ((x.hi >> j) & 1u) * 2u;
        const uint32_t q = (x.qw >> j) & 1u;
        const uint32_t n0 = pre + q, n1 = pre + 1u - q;
        K0 = tab_s + 4u * n0; K1 = tab_s + 4u * n1; D0 = 40u - 20u * n0; D1 = 40u - 20u * n1;
    };
    if (MODE >= 10) {
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
    } else if (MODE == 0 || (MODE >= 2 && MODE < 10)) {
        uint32_t K0, K1, D0, D1;
        consts(cur, 0, K0, K1, D0, D1);
        uint32_t A0 = lds_u32(P0 + K0), A1 = lds_u32(P1 + K1);
        for (int wi = 0; wi < n_words; ++wi) {
            Word nx{cur.lo * 3u + lcg(s), cur.hi ^ lcg(s), cur.qw + lcg(s)};
            uint4 blk = drw[lane], blk_next = drw[32 + lane];
            uint32_t Rw = 0, K0n = 0, K1n = 0, D0n = 0, D1n = 0;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int kk = j & 3;
                if (kk == 0 && j > 0) { blk = blk_next; if (j < 28) blk_next = drw[((j >> 2) + 1) * 32 + lane]; }
                const uint32_t u = min(kk == 0 ? blk.x : kk == 1 ? blk.y : kk == 2 ? blk.z : blk.w, 0xFFFFFFFEu);
                if (MODE == 3 || MODE == 4 || MODE == 6 || MODE == 7) { K0n = tab_s + 4u * (j & 3); K1n = tab_s + 4u * ((j + 1) & 3); D0n = 40u - 20u * (j & 3); D1n = 40u - 20u * ((j + 1) & 3); }
                else if (j < 31) consts(cur, j + 1, K0n, K1n, D0n, D1n); else consts(nx, 0, K0n, K1n, D0n, D1n);
                const uint32_t o0 = ap ? P1 + K0n : P0 + K0n;
                const uint32_t o1 = ap ? P1 + D1 + K1n : P0 + D0 + K1n;
                uint32_t A0n, A1n;
                bool acc;
                if (MODE == 2 || MODE == 3) { A0n = (o0 * 0x9E3779B1u) | 0x80000000u; A1n = (o1 * 0x85EBCA6Bu) | 0x80000000u; }
                else if (MODE == 5) { A0n = A0; A1n = A1; }
                else if (MODE == 6 || MODE == 8) {
                    // loads, then the compare's input through a volatile move
                    A0n = lds_u32(o0); A1n = lds_u32(o1);
                }
                else if (MODE == 7 || MODE == 9) { A0n = 0; A1n = 0; }
                else { A0n = lds_u32(o0); A1n = lds_u32(o1); }
                if (MODE == 7 || MODE == 9) {
                    const uint32_t A = ap ? A1 : A0;
                    uint32_t a32;
                    asm volatile("{\n\t.reg .pred p;\n\tld.shared.u32 %0, [%3];\n\tld.shared.u32 %1, [%4];\n\t"
                                 "setp.lt.u32 p, %5, %6;\n\tselp.u32 %2, 1, 0, p;\n\t}"
                                 : "=r"(A0n), "=r"(A1n), "=r"(a32) : "r"(o0), "r"(o1), "r"(u), "r"(A));
                    acc = a32 != 0u;
                } else if (MODE == 6 || MODE == 8) {
                    uint32_t A = ap ? A1 : A0;
                    asm volatile("mov.b32 %0, %0;" : "+r"(A));
                    acc = u < A;
                } else {
                    const uint32_t A = ap ? A1 : A0;
                    acc = u < A;
                }
                if (MODE == 5) { ap = acc; Rw ^= acc ? (1u << j) : 0u; continue; }
                const uint32_t nP0 = ap ? P1 : P0, nP1 = ap ? P1 + D1 : P0 + D0;
                A0 = A0n; A1 = A1n; P0 = nP0; P1 = nP1; D0 = D0n; D1 = D1n;
                Rw ^= acc ? (1u << j) : 0u;
                ap = acc;
            }
            Racc += Rw;
            cur = nx;
        }
    } else {
        // 2-deep: at site j the four thresholds of site j+2 are loaded, their offsets
        // resolved by site j-1's decision; site j+1's four are reduced to two with
        // site j's decision; site j+2 picks one of two with site j+1's.
        // State entering site j: ap = acc(j-1); Pb = bin20 before site j given ap
        // resolved (known); Dj0/Dj1: site j's bin change for left old/flipped.
        uint32_t Kj0, Kj1, Dj0, Dj1, Kn0, Kn1, Dn0, Dn1;
        consts(cur, 0, Kj0, Kj1, Dj0, Dj1);
        consts(cur, 1, Kn0, Kn1, Dn0, Dn1);
        uint32_t Pb = P0;
        // site 0: its two candidates (acc(-1) = 0 known: take the left-old column)
        uint32_t B0 = lds_u32(Pb + Kj0), B1 = B0;            // pair for site j (by acc(j-1))
        // site 1: four candidates by (acc0): bin Pb or Pb+Dj0; column by acc0
        uint32_t C00 = lds_u32(Pb + Kn0), C01 = lds_u32(Pb + Dj0 + Kn1);
        uint32_t C10 = C00, C11 = C01;                         // (acc(j-1)=1 impossible for site 0)
        for (int wi = 0; wi < n_words; ++wi) {
            Word nx{cur.lo * 3u + lcg(s), cur.hi ^ lcg(s), cur.qw + lcg(s)};
            uint4 blk = drw[lane], blk_next = drw[32 + lane];
            uint32_t Rw = 0;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int kk = j & 3;
                if (kk == 0 && j > 0) { blk = blk_next; if (j < 28) blk_next = drw[((j >> 2) + 1) * 32 + lane]; }
                const uint32_t u = min(kk == 0 ? blk.x : kk == 1 ? blk.y : kk == 2 ? blk.z : blk.w, 0xFFFFFFFEu);
                // site j+2 constants
                uint32_t Km0, Km1, Dm0, Dm1;
                if (j < 30) consts(cur, j + 2, Km0, Km1, Dm0, Dm1); else consts(nx, j - 30, Km0, Km1, Dm0, Dm1);
                // bin before site j (known: ap resolved), site j's change given ap
                const uint32_t Dj = ap ? Dj1 : Dj0;
                // loads for site j+2 by (acc j, acc j+1): bin = Pb + acc_j*Dj + acc_{j+1}*Dn(acc_j)
                const uint32_t E00 = lds_u32(Pb + Km0);
                const uint32_t E10 = lds_u32(Pb + Dj + Km0);
                const uint32_t E01 = lds_u32(Pb + Dn0 + Km1);
                const uint32_t E11 = lds_u32(Pb + Dj + Dn1 + Km1);
                // decide site j
                const uint32_t A = ap ? B1 : B0;
                const bool acc = u < A;
                // site j+1's pair by acc_j; site j+2's quadruple stays keyed by (acc_j, acc_j+1)
                const uint32_t nB0 = acc ? C10 : C00, nB1 = acc ? C11 : C01;
                Pb = acc ? Pb + Dj : Pb;
                B0 = nB0; B1 = nB1;
                C00 = E00; C10 = E10; C01 = E01; C11 = E11;
                // shift constants: site j+1 becomes current
                Dj0 = Dn0; Dj1 = Dn1; Dn0 = Dm0; Dn1 = Dm1;
                Rw ^= acc ? (1u << j) : 0u;
                ap = acc;
            }
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
    cudaFuncSetAttribute(k<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k<7>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k<9>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k<10>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k<11>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const char *names[] = {"1-deep", "2-deep", "1-deep, ALU thresholds", "ALU thresholds, fixed consts",
                           "loads, fixed consts", "accept chain only", "fixed consts, volatile-mov fence",
                           "fixed consts, loads+compare in one asm", "real consts, volatile-mov fence",
                           "real consts, loads+compare in one asm", "byte-parallel consts (kernel)",
                           "byte-parallel, 16 chains per warp", "byte-parallel, 8 chains per warp"};
    for (int mode = 0; mode < 13; ++mode)
        for (int rep = 0; rep < 1; ++rep) {
            switch (mode) {
            case 0: k<0><<<blocks, 32, smem>>>(gtab, n_words, out, cyc); break;
            case 1: k<1><<<blocks, 32, smem>>>(gtab, n_words, out, cyc); break;
            case 2: k<2><<<blocks, 32, smem>>>(gtab, n_words, out, cyc); break;
            case 3: k<3><<<blocks, 32, smem>>>(gtab, n_words, out, cyc); break;
            case 4: k<4><<<blocks, 32, smem>>>(gtab, n_words, out, cyc); break;
            case 5: k<5><<<blocks, 32, smem>>>(gtab, n_words, out, cyc); break;
            case 6: k<6><<<blocks, 32, smem>>>(gtab, n_words, out, cyc); break;
            case 7: k<7><<<blocks, 32, smem>>>(gtab, n_words, out, cyc); break;
            case 8: k<8><<<blocks, 32, smem>>>(gtab, n_words, out, cyc); break;
            case 9: k<9><<<blocks, 32, smem>>>(gtab, n_words, out, cyc); break;
            case 10: k<10><<<blocks, 32, smem>>>(gtab, n_words, out, cyc); break;
            case 11: k<11><<<blocks, 32, smem>>>(gtab, n_words, out, cyc); break;
            default: k<12><<<blocks, 32, smem>>>(gtab, n_words, out, cyc); break;
            }
            if (cudaDeviceSynchronize() != cudaSuccess) { printf("error\n"); return 1; }
            long long c[blocks]; cudaMemcpy(c, cyc, sizeof c, cudaMemcpyDeviceToHost);
            double m = 0; for (int i = 0; i < blocks; ++i) m += c[i];
            printf("mode %d (%s): %.1f cycles/site\n", mode, names[mode], m / blocks / (n_words * 32.0));
        }
    return 0;
}
