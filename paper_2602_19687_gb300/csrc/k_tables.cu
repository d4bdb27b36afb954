// Per-cell bilinear coefficients of the opacity tables (Sect. 3), built once
// per table load. For species s and the (T, p) cell (it, ip) with corner
// values v_ab = log10 sigma_s(T_{it+a}, p_{ip+b}, nu) (BF16 residual + row
// offset, or FP32), the interpolated exponent in log2 units is
//   e = c0 + wp c1 + wt (c2 + wp c3),
//   c0 = L v00, c1 = L (v01 - v00), c2 = L (v10 - v00),
//   c3 = L ((v11 - v10) - (v01 - v00)),  L = log2(10),
// identical to bilinear interpolation with weights (1-wt)(1-wp), (1-wt) wp,
// wt (1-wp), wt wp. Species slot s = h SP/2 + j of a wavenumber pair is
// read by the lane of half h of the pair; its two float4 (c0, c0', c1, c1')
// and (c2, c2', c3, c3') (primes: the pair's second wavenumber) sit at
// [cell][j][c][pair][h], so that for fixed (j, c) the lanes of a warp read
// consecutive float4. Slots s >= S stay zero (the caller clears the table).
#include "internal.cuh"

namespace es {

namespace {

template <bool BF16>
__device__ __forceinline__ float table_value(const Model &m, size_t row, int n) {
    const size_t idx = row * (size_t)m.Np + n;
    const float q = BF16 ? __uint_as_float(((uint32_t)m.tab16[idx]) << 16) : m.tab32[idx];
    return q + m.row_off[row];
}

template <bool BF16>
__global__ void k_build_coef(Model m, float4 *coef) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const int cs = blockIdx.y;                       // cell * S + s
    if (n >= m.Np) return;
    const int s = cs % m.S, cell = cs / m.S;
    const int it = cell / (m.NP - 1), ip = cell % (m.NP - 1);
    const size_t row = ((size_t)s * m.NT + it) * m.NP + ip;
    const float v00 = table_value<BF16>(m, row, n), v01 = table_value<BF16>(m, row + 1, n);
    const float v10 = table_value<BF16>(m, row + m.NP, n), v11 = table_value<BF16>(m, row + m.NP + 1, n);
    const float l = (float)LOG2_10, d0 = v01 - v00;
    const int spl = m.SP >> 1, h = s / spl, j = s % spl;
    const size_t np2 = (size_t)(m.Np >> 1);
    const size_t i0 = ((((size_t)cell * spl + j) * 2 + 0) * np2 + (n >> 1)) * 2 + h;
    const size_t i1 = i0 + 2 * np2;   // c = 1
    float *o0 = reinterpret_cast<float *>(coef + i0) + (n & 1);
    float *o1 = reinterpret_cast<float *>(coef + i1) + (n & 1);
    o0[0] = l * v00;
    o0[2] = l * d0;
    o1[0] = l * (v10 - v00);
    o1[2] = l * ((v11 - v10) - d0);
}

}  // namespace

int launch_build_coef(const Model &m, float4 *coef, cudaStream_t st) {
    dim3 grid((m.Np + 255) / 256, (m.NT - 1) * (m.NP - 1) * m.S);
    if (m.bf16) k_build_coef<true><<<grid, 256, 0, st>>>(m, coef);
    else k_build_coef<false><<<grid, 256, 0, st>>>(m, coef);
    return 1;
}

}  // namespace es
