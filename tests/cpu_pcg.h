// CPU stand-in for the library's device-scalar PCG kernels (k_init,
// k_update, k_dir of dev_pcg.cuh) with the same scalar layout
// sc[3k + {0, 1, 2}] = (rz_k, pq_k, rr_k), for host builds that run the
// library's control code (dpcg_control.h and the controls built on it).
// Vectors in T; each product rounded to T and the sum taken in double, as
// the device's per-thread partials (one element per thread at these sizes)
// and FP64 block sums do.  Test code only.
#pragma once

#include <cstring>
#include <functional>
#include <string>
#include <vector>

template <typename T>
struct CpuPcg {
    int64_t n;
    std::function<void(const T *, T *, double *)> apply;  // y = A x; *dot += (x, y) when dot
    const T *dinv, *b;
    T *u;
    int maxit;
    std::vector<T> r, z, p, q;
    std::vector<double> sc;
    std::string err;

    int start(double *rz0, double *rr0, double *bb)
    {
        sc.assign(3 * ((size_t)maxit + 2), 0.0);
        r.assign(n, (T)0), z.assign(n, (T)0), p.assign(n, (T)0), q.assign(n, (T)0);
        apply(u, q.data(), nullptr);
        double b2 = 0;
        for (int64_t i = 0; i < n; ++i) {
            r[i] = b[i] - q[i];
            z[i] = dinv[i] * r[i];
            p[i] = z[i];
            sc[0] += (double)(T)(r[i] * z[i]);
            sc[2] += (double)(T)(r[i] * r[i]);
            b2 += (double)(T)(b[i] * b[i]);
        }
        *rz0 = sc[0], *rr0 = sc[2], *bb = b2;
        return 0;
    }
    bool halt = false;

    int iterate(int k0, int k1)
    {
        for (int k = k0; k < k1; ++k) {
            double *sck = &sc[3 * (size_t)k], *sck1 = &sc[3 * ((size_t)k + 1)];
            apply(p.data(), q.data(), &sck[1]);
            if (halt || !(sck[1] > 0.0)) {  // truncated: carry the scalars, keep the iterate
                sck1[0] = sck[0];
                sck1[2] = sck[2];
                halt = true;
                continue;
            }
            const T alpha = (T)(sck[0] / sck[1]);
            for (int64_t i = 0; i < n; ++i) {
                u[i] += alpha * p[i];
                r[i] = r[i] - alpha * q[i];
                z[i] = dinv[i] * r[i];
                sck1[0] += (double)(T)(r[i] * z[i]);
                sck1[2] += (double)(T)(r[i] * r[i]);
            }
            const T beta = sck[0] > 0.0 ? (T)(sck1[0] / sck[0]) : (T)0;
            for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        }
        return 0;
    }
    int read(int k0, int k1, double *hs)
    {
        std::memcpy(hs, &sc[3 * (size_t)k0], sizeof(double) * 3 * (size_t)(k1 - k0 + 1));
        return 0;
    }
    void fail(const char *what) { err = what; }
};
