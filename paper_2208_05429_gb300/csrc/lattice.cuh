// lattice.cuh -- the D3Q15 and D3Q27 velocity sets (host and device,
// compile-time), beside the D3Q19 set of d3q19.cuh.
//
// The three cubic sets the paper's dependency guard covers (Sec. 4.1) share
// one construction here: direction 0 is the rest vector; directions 1 .. H,
// H = (q - 1) / 2, are the admitted vectors of {-1, 0, 1}^3 whose first
// non-zero component is -1 (the half of the neighbours the swap scheme
// streams to, Sec. 3), taken in lexicographic (cx, cy, cz) order; direction
// i + H is the opposite of i.  D3Q15 admits |c|^2 in {0, 1, 3} (rest, six
// faces, eight corners; w = 2/9, 1/9, 1/72), D3Q27 every vector (w = 8/27,
// 2/27, 1/54, 1/216 for |c|^2 = 0 .. 3, the product of three D1Q3 sets).
// c_s^2 = 1/3 on both.
#pragma once

namespace lbm {

template <int QN>
struct DQ {
    static_assert(QN == 15 || QN == 27, "D3Q15 or D3Q27");
    static constexpr int Q = QN;
    static constexpr int H = (QN - 1) / 2;

    __host__ __device__ static constexpr bool admitted(int a, int b, int c)
    {
        return QN == 27 || a * a + b * b + c * c != 2;
    }
    // vector code (cx + 1) * 9 + (cy + 1) * 3 + (cz + 1) of the k-th vector
    // (k = 1 .. H) of the backward half
    __host__ __device__ static constexpr int half_code(int k)
    {
        int m = 0;
        for (int a = -1; a <= 1; ++a)
            for (int b = -1; b <= 1; ++b)
                for (int c = -1; c <= 1; ++c) {
                    const int first = a != 0 ? a : (b != 0 ? b : c);
                    if (first == -1 && admitted(a, b, c) && ++m == k) return (a + 1) * 9 + (b + 1) * 3 + (c + 1);
                }
        return 13;
    }
    __host__ __device__ static constexpr int code(int i)
    {
        return i == 0 ? 13 : (i <= H ? half_code(i) : 26 - half_code(i - H));
    }
    __host__ __device__ static constexpr int cx(int i) { return code(i) / 9 - 1; }
    __host__ __device__ static constexpr int cy(int i) { return code(i) / 3 % 3 - 1; }
    __host__ __device__ static constexpr int cz(int i) { return code(i) % 3 - 1; }
    __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : (i <= H ? i + H : i - H); }
    __host__ __device__ static constexpr int csq(int i) { return cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i); }
    __host__ __device__ static constexpr double wgt(int i)
    {
        if constexpr (QN == 15) {
            return csq(i) == 0 ? 2.0 / 9.0 : (csq(i) == 1 ? 1.0 / 9.0 : 1.0 / 72.0);
        } else {
            return csq(i) == 0 ? 8.0 / 27.0 : csq(i) == 1 ? 2.0 / 27.0 : csq(i) == 2 ? 1.0 / 54.0 : 1.0 / 216.0;
        }
    }
};

}  // namespace lbm
