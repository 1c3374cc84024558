// pic_device.cuh -- device-side types and helpers of the GB300 r-z PIC/MCC library.
//
// Particle store: per species, two buffers (read / write).  A particle's state
// is two 4-vectors and its id: pa = (fr, fz, vr, vt), pb = (vz, ar, at, az) --
// one 16-byte load or store each in FP32 (32 bytes in FP64) -- and the 64-bit
// id in an array of its own.  Positions are cell-relative:
// the cell is implied by the bin the particle sits in, (fr, fz) in [0,1) is
// the offset inside it in cell units, so FP32 keeps ~1e-7 of a cell at any
// radius.  Bins are cells in tile-major order: TX x TY cells per tile, the
// tile's bins contiguous, so one CTA reads one tile's particles contiguously.
// Each bin has room for its particles plus slack; particles that do not fit
// their new bin go to an overflow region at the end of the buffer.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pic {

constexpr int kSpecies = 2;
constexpr int kHalo = 4;          // deposit tile halo, cells
constexpr int kThreads = 256;     // particle kernel CTA size
constexpr int kOvfCtas = 64;      // CTAs that sweep the overflow region

// Counter slots (u64) written by the particle kernel.
enum Counter : int {
  CNT_ABS = 0,        // [species*3 + kind], kind 0 powered, 1 grounded, 2 surface
  CNT_COLL = 6,       // [species*3 + process]
  CNT_BORN = 12,      // [species]
  CNT_OVERFLOW = 14,  // particles dropped because the overflow region was full
  CNT_OUTSIDE = 15,   // particles read from the store outside the plasma
  CNT_ABSW = 16,      // weighted particles: absorbed macro weight [species*3 + kind],
                      // in units of 2^-32 of the species' macro weight
  CNT_SPLIT = 22,     // [species] particles split near the axis
  CNT_N = 24
};

// Fixed-point unit of weighted absorption tallies (CNT_ABSW, surface charge).
constexpr double kCreditOne = 4294967296.0;  // 2^32

// Scalars (double) shared by the circuit, assembly and diagnostics kernels.
enum Scalar : int {
  SC_T = 0, SC_UE, SC_QE, SC_CEQ, SC_ICONV, SC_ICCP,
  SC_Y0 = 6,                                  // 6 circuit states
  SC_ITERS = 12, SC_RELRES, SC_STATUS,
  SC_DFT_RE, SC_DFT_IM, SC_I1_RE, SC_I1_IM,
  SC_IONQ = 19,                               // 3 sums over the window
  SC_IONCUR = 22,                             // 3 window averages
  SC_WINDOWS = 25, SC_WINCOUNT, SC_CEQ_GAUSS, SC_BNORM, SC_ENERGY,
  SC_CW_RE = 32,                              // 5 first-harmonic DFT sums of the circuit
  SC_CW_IM = 37,                              //   waveforms (U_s, I_1, U_in, U_E, I_ccp)
  SC_CP = 42,                                 // 6 sums of the element powers
  SC_CDC = 48,                                // 2 sums of U_E and I_ccp (DC parts)
  SC_COUT = 50,                               // 18 results of the last window (PIC_DIAG_CIRCUIT)
  SC_N = 72
};

struct BinMeta {
  int ovf_base;   // first overflow slot
  int ovf_n;      // overflow particles claimed (may exceed room; excess dropped)
  long long total;
};

// Four values of a particle's state, aligned for one vector access.
template <typename T> struct Vec4;
template <> struct alignas(16) Vec4<float> { float x, y, z, w; };
template <> struct alignas(32) Vec4<double> { double x, y, z, w; };

template <typename T>
struct StoreView {
  Vec4<T> *pa;    // (fr, fz, vr, vt)
  Vec4<T> *pb;    // (vz, ar, at, az)
  unsigned long long *id;
  T *w;           // weight ratios in (0, 1] (weighted handles only)
  int *cell;      // only meaningful in the overflow region
  int *start;     // [nbins] first slot of each bin
  int *cap;       // [nbins] room of each bin
  int *fill;      // [nbins] particles whose cell is this bin (incl. overflowed ones)
  BinMeta *meta;
  int capacity;
};

// Mapping between cells (i, j) and bins.
struct BinMap {
  int nr, nz, TX, TY, ntx, nty;
  __host__ __device__ __forceinline__ int bin(int i, int j) const {
    int tx = i / TX, ty = j / TY;
    return ((ty * ntx + tx) * TY + (j - ty * TY)) * TX + (i - tx * TX);
  }
  __host__ __device__ __forceinline__ void cell(int b, int &i, int &j) const {
    int per = TX * TY;
    int t = b / per, l = b - t * per;
    int ty = t / ntx, tx = t - ty * ntx;
    j = ty * TY + l / TX;
    i = tx * TX + (l - (l / TX) * TX);
  }
  __host__ __device__ __forceinline__ int nbins() const { return ntx * nty * TX * TY; }
  __host__ __device__ __forceinline__ int ntiles() const { return ntx * nty; }
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds; each round
// multiplies words 0 and 2 by two fixed 32-bit constants, swaps in the high
// halves xor'ed with words 1, 3 and the round key; keys advance by Weyl steps.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ void philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                  uint32_t k0, uint32_t k1, uint32_t out[4]) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
#ifdef __CUDA_ARCH__
    uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
#else
    uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0, hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
    uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Top 24 bits as a uniform in [0,1): exact in FP32 and FP64.
template <typename T>
__device__ __forceinline__ T unif24(uint32_t x) {
  return (T)(x >> 8) * (T)5.9604644775390625e-8;  // 2^-24
}

}  // namespace pic
