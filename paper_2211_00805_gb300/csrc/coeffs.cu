// Host FP64 Chebyshev coefficients of the heat kernel (Sec. 3.5).
//
// exp(-t L) = exp(-t (Id - P)) and, with the generating function of the modified Bessel
// functions, exp(t y) = I_0(t) + 2 sum_{k>=1} I_k(t) T_k(y) for y in [-1, 1].  Hence
//     exp(-t L) = sum_k c_k T_k(P),  c_0 = e^{-t} I_0(t),  c_k = 2 e^{-t} I_k(t)  (k >= 1),
// the paper's expansion in T_k(L - Id) = (-1)^k T_k(P) with the alternating signs absorbed.
//
// The scaled values e^{-t} I_k(t) come from Miller's backward recurrence: the sequence
// I_{k-1}(t) = I_{k+1}(t) + (2k / t) I_k(t) is run downwards from an index N far above K and t
// with arbitrary starting values; it converges to a multiple of the true I_k, and the multiple is
// fixed by the identity e^{t} = I_0(t) + 2 sum_{k>=1} I_k(t) (all terms positive, no cancellation).
#include <math.h>

#include <vector>

#include "gs_internal.cuh"

void gs_heat_coefficients(double t, int K, double* c)
{
    const int N = K + 40 + (int)(t + 10.0 * sqrt(t + 1.0));
    std::vector<double> f((size_t)N + 2, 0.0);
    f[N + 1] = 0.0;
    f[N] = 1.0;
    for (int k = N; k >= 1; --k) {
        f[k - 1] = f[k + 1] + (2.0 * k / t) * f[k];
        if (f[k - 1] > 1e250) {                 // keep the unnormalised sequence in range
            for (int j = k - 1; j <= N + 1; ++j) f[j] *= 1e-250;
        }
    }
    double tail = 0.0;                          // 2 sum_{k>=1} f_k, smallest terms first
    for (int k = N; k >= 1; --k) tail += 2.0 * f[k];
    const double norm = f[0] + tail;            // proportional to e^{t}
    c[0] = f[0] / norm;
    for (int k = 1; k <= K; ++k) c[k] = 2.0 * f[k] / norm;
}
