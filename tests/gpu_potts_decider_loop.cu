// Replica of the 8-Potts slot decider's loop (32 sites of a ring slot as one unrolled
// block), timed alone on one warp per block (test infrastructure: it measures the
// chain-latency bound of the 8-Potts sweeps that the benchmark reports; it is not part
// of the library).
//
// Per word of 4 sites it reads the draws and the producer's records (proposals, column
// counts, old spins) and the upper neighbour word, corrects the column counts
// byte-parallel, and per site extracts the two column bytes, forms the two bin changes,
// selects the bin and its change with the previous decision, loads the two candidate
// thresholds of the next site before the current site is decided, then select ->
// compare; the row's last site and first site get their corrections as in the kernel.
// Output: cycles per site (clock64).  Thresholds are random; the rows of the NB_EDGE
// lowest and highest bins are 0 (never accept), so every bin, including the speculative
// one of the next site, stays inside the table.
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>
constexpr int NBINS = 2049, NCOL = 9, NB_EDGE = 8, ROWW = 8;  // 8-Potts 32 x 32: 8 words per row

__device__ __forceinline__ uint32_t lds_u32(uint32_t a)
{
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ uint32_t byte_of(uint32_t x, int k) { return __byte_perm(x, 0u, 0x4440u | (uint32_t)k); }
__device__ __forceinline__ uint32_t nz8(uint32_t x) { return ((x + 0x7F7F7F7Fu) >> 7) & 0x01010101u; }
__device__ __forceinline__ uint32_t lcg(uint32_t &s) { s = s * 1664525u + 1013904223u; return s; }

struct Word {
    uint4 u;
    uint32_t R, SN, C0, C1;
};

__global__ void __launch_bounds__(32) k(const uint32_t *gtab, int n_slots, uint32_t *out, long long *cyc)
{
    extern __shared__ uint32_t sm[];
    uint32_t *tab = sm;                                                   // NBINS * NCOL
    uint4 *ring = reinterpret_cast<uint4 *>(sm + ((NBINS * NCOL + 3) & ~3));  // [16][32]: draws, records per word
    uint32_t *lat = reinterpret_cast<uint32_t *>(ring + 16 * 32);         // [2 rows][8][32]
    for (int i = threadIdx.x; i < NBINS * NCOL; i += 32) tab[i] = gtab[i];
    const int lane = threadIdx.x;
    uint32_t s = 777u + 7919u * lane;
    for (int w = 0; w < ROWW; ++w) {
        // spins 0..7 per byte, proposals different from them, producer counts 2..6 (the
        // upper-neighbour and row-end corrections, +-1 each, keep every column count in
        // 0..8, so every table address stays inside its bin's row)
        uint32_t R = 0, SN = 0, c0 = 0, c1 = 0;
        for (int b = 0; b < 4; ++b) {
            const uint32_t r = lcg(s) >> 29, sn = (r + 1 + (lcg(s) >> 29) % 7) & 7u;
            R |= r << (8 * b);
            SN |= sn << (8 * b);
            c0 |= (2u + (lcg(s) >> 29) % 5) << (8 * b);
            c1 |= (2u + (lcg(s) >> 29) % 5) << (8 * b);
        }
        ring[(2 * w) * 32 + lane] = make_uint4(lcg(s), lcg(s), lcg(s), lcg(s));
        ring[(2 * w + 1) * 32 + lane] = make_uint4(SN, c0, c1, R);
        lat[w * 32 + lane] = R;
        lat[(ROWW + w) * 32 + lane] = (R ^ 0x01010101u) & 0x07070707u;
    }
    __syncwarp();
    const uint32_t tab_s = (uint32_t)__cvta_generic_to_shared(tab);
    uint32_t P0 = tab_s + 36u * (uint32_t)(NBINS / 2 + (lane & 7)), P1 = P0;
    bool ap = false;
    uint32_t first_new = 0u, acc_all = 0u;
    auto columns = [](Word &x, const uint4 &r1, uint32_t U) {
        x.R = r1.w;
        x.SN = r1.x;
        const uint32_t d = nz8(U ^ r1.x) - nz8(U ^ r1.w);
        x.C0 = r1.y + d;
        x.C1 = r1.z + d;
    };
    long long t0 = clock64();
    Word cur;
    cur.u = ring[lane];
    columns(cur, ring[32 + lane], lat[ROWW * 32 + lane]);
    uint32_t K0 = byte_of(cur.C0, 0), K1 = byte_of(cur.C1, 0);
    uint32_t D0 = 36u * K0 - 144u, D1 = 36u * K1 - 144u;
    uint32_t A0 = lds_u32(P0 + 4u * K0), A1 = lds_u32(P1 + 4u * K1);
    for (int sl = 0; sl < n_slots; ++sl) {
        const int up = (sl & 1) ? 0 : ROWW;  // rows alternate: the other one is "above"
        const int kr = ROWW - up;
        uint32_t Fm = 0u;
        Word nx = cur;
        uint4 nr1 = make_uint4(0u, 0u, 0u, 0u);
        uint32_t nU = 0u;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const int w = j >> 2, kk = j & 3;
            if (kk == 0) {
                const int w1 = (w + 1) & 7;  // the next word (the next slot's first after word 7)
                nx.u = ring[(2 * w1) * 32 + lane];
                nr1 = ring[(2 * w1 + 1) * 32 + lane];
                nU = lat[((w < 7 ? up : kr) + w1) * 32 + lane];
            }
            if (kk == 1) columns(nx, nr1, nU);
            if (w == 7 && kk == 1) {
                // the row's last site: its right neighbour is site 0 of the row, updated
                const uint32_t s3 = cur.R >> 24, sn3 = cur.SN >> 24;
                const uint32_t dK = ((first_new == s3 ? 1u : 0u) - (first_new == sn3 ? 1u : 0u)) << 24;
                cur.C0 += dK;
                cur.C1 += dK;
            }
            const uint32_t Kn0 = kk < 3 ? byte_of(cur.C0, kk + 1) : byte_of(nx.C0, 0);
            const uint32_t Kn1 = kk < 3 ? byte_of(cur.C1, kk + 1) : byte_of(nx.C1, 0);
            const uint32_t Dn0 = 36u * Kn0 - 144u, Dn1 = 36u * Kn1 - 144u;
            const uint32_t Pb = ap ? P1 : P0;
            const uint32_t PbD = Pb + (ap ? D1 : D0);
            const uint32_t A0n = lds_u32(Pb + 4u * Kn0), A1n = lds_u32(PbD + 4u * Kn1);
            const uint32_t u = min(kk == 0 ? cur.u.x : kk == 1 ? cur.u.y : kk == 2 ? cur.u.z : cur.u.w, 0xFFFFFFFEu);
            const bool acc = u < (ap ? A1 : A0);
            Fm |= acc ? (0xFFu << (8 * kk)) : 0u;
            if (j == 0) first_new = acc ? (cur.SN & 0xFFu) : (cur.R & 0xFFu);
            P0 = Pb;
            P1 = PbD;
            D0 = Dn0;
            D1 = Dn1;
            A0 = A0n;
            A1 = A1n;
            ap = acc;
            if (kk == 3) {
                lat[(kr + w) * 32 + lane] = (cur.R & ~Fm) | (cur.SN & Fm);
                acc_all += Fm;
                Fm = 0u;
                cur = nx;
            }
        }
    }
    long long t1 = clock64();
    out[blockIdx.x * 32 + lane] = acc_all ^ P0 ^ P1;
    if (lane == 0) cyc[blockIdx.x] = t1 - t0;
}

int main()
{
    const int n_slots = 4096, blocks = 32;
    uint32_t *h = new uint32_t[NBINS * NCOL];
    uint32_t s = 1;
    for (int b = 0; b < NBINS; ++b)
        for (int c = 0; c < NCOL; ++c) {
            s = s * 1664525u + 1013904223u;
            h[b * NCOL + c] = (b < NB_EDGE || b >= NBINS - NB_EDGE) ? 0u : s;
        }
    uint32_t *gtab, *out;
    long long *cyc;
    cudaMalloc(&gtab, NBINS * NCOL * 4);
    cudaMalloc(&out, blocks * 32 * 4);
    cudaMalloc(&cyc, blocks * 8);
    cudaMemcpy(gtab, h, NBINS * NCOL * 4, cudaMemcpyHostToDevice);
    const size_t smem = ((NBINS * NCOL + 3) & ~3) * 4 + 16 * 32 * 16 + 2 * ROWW * 32 * 4;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<blocks, 32, smem>>>(gtab, n_slots, out, cyc);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        printf("error\n");
        return 1;
    }
    long long c[blocks];
    cudaMemcpy(c, cyc, sizeof c, cudaMemcpyDeviceToHost);
    double m = 0;
    for (int i = 0; i < blocks; ++i) m += c[i];
    printf("potts decider loop: %.1f cycles/site\n", m / blocks / (n_slots * 32.0));
    delete[] h;
    return 0;
}
