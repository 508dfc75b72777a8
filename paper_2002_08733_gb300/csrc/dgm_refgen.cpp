// Build-time generator of the straight-line reference operators.
//
// Runs the library's own reference-matrix construction (dgm_refmats.cpp) for
// every supported degree and writes a CUDA header with, per degree p:
//   TraceOp<p, f>::apply(v, acc)       acc[m] = sum_l R_f[m][l] v[l]
//   LiftOp<p, f>::apply(g, stride, acc) acc[l] += sum_m R_f[m][l] g[m]
//   DerivOp<p, a>::apply(v, stride, s, acc) acc[l] += s sum_m S_a[l][m] v[m]
// as unrolled code whose coefficients are literals, emitting only the
// entries that are not zero.  Many entries of the geometry-free operators of
// Eq. (matrix_free_curl) vanish exactly for the collapsed modal basis
// (S_a[l][m] = 0 unless deg l < deg m; on the face x = 0 the trace of mode
// (i,j,k) is a single face mode), so the kernels issue only the FMAs that
// contribute.  Entries below 1e-13 of the matrix's largest entry are
// round-off of exact zeros and are dropped.  Host copies of the full
// matrices are emitted too, so that the library can check at plan creation
// that the compiled operators match the matrices it builds at run time.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "dgm_internal.h"

using namespace dgm;

static void lit(FILE* f, double v) { std::fprintf(f, "R(%.17g)", v); }

int main(int argc, char** argv) {
    if (argc < 2) {
        std::fprintf(stderr, "usage: %s out.cuh\n", argv[0]);
        return 2;
    }
    FILE* f = std::fopen(argv[1], "w");
    if (!f) return 1;
    std::fprintf(f, "// Generated by dgm_refgen.cpp at build time; do not edit.\n#pragma once\n\n");
    std::fprintf(f, "namespace dgm {\n\n");
    std::fprintf(f, "// fused multiply-add used by the operators (overloaded per real type)\n");
    std::fprintf(f, "__device__ __forceinline__ float fmaa(float a, float b, float c) { return fmaf(a, b, c); }\n");
    std::fprintf(f, "__device__ __forceinline__ double fmaa(double a, double b, double c) { return fma(a, b, c); }\n\n");
    std::fprintf(f, "template <int P, int F> struct TraceOp;\ntemplate <int P, int F> struct LiftOp;\n");
    std::fprintf(f, "template <int P, int A> struct DerivOp;\ntemplate <int P, int A> struct DerivTOp;\n");
    std::fprintf(f, "template <int P> struct RefNnz;\n\n");
    for (int p = 1; p <= PMAX; ++p) {
        std::vector<double> S, Rm;
        std::string err;
        if (build_refmats(p, S, Rm, err)) {
            std::fprintf(stderr, "p=%d: %s\n", p, err.c_str());
            return 1;
        }
        const int N = nmodes(p), NF = nfmodes(p);
        double smax = 0, rmax = 0;
        for (double v : S) smax = std::fmax(smax, std::fabs(v));
        for (double v : Rm) rmax = std::fmax(rmax, std::fabs(v));
        auto sv = [&](int a, int l, int m) {
            double v = S[(a * N + l) * N + m];
            return std::fabs(v) > 1e-13 * smax ? v : 0.0;
        };
        auto rv = [&](int fc, int m, int l) {
            double v = Rm[(fc * NF + m) * N + l];
            return std::fabs(v) > 1e-13 * rmax ? v : 0.0;
        };
        int nnzS = 0, nnzR = 0;
        for (int fc = 0; fc < 4; ++fc) {
            std::fprintf(f, "template <> struct TraceOp<%d, %d> {\n  template <typename R>\n"
                            "  __device__ static __forceinline__ void apply(const R* v, R* acc) {\n", p, fc);
            for (int m = 0; m < NF; ++m) {
                bool first = true;
                for (int l = 0; l < N; ++l) {
                    double c = rv(fc, m, l);
                    if (c == 0.0) continue;
                    ++nnzR;
                    if (first) {
                        std::fprintf(f, "    acc[%d] = ", m);
                        lit(f, c);
                        std::fprintf(f, " * v[%d];", l);
                        first = false;
                    } else {
                        std::fprintf(f, " acc[%d] = fmaa(", m);
                        lit(f, c);
                        std::fprintf(f, ", v[%d], acc[%d]);", l, m);
                    }
                }
                if (first) std::fprintf(f, "    acc[%d] = R(0);", m);
                std::fprintf(f, "\n");
            }
            std::fprintf(f, "  }\n};\n");
            std::fprintf(f, "template <> struct LiftOp<%d, %d> {\n  template <typename R, int LO = 0, int HI = %d>\n"
                            "  __device__ static __forceinline__ void apply(const R* g, int stride, R* acc) {\n",
                         p, fc, N);
            for (int m = 0; m < NF; ++m) {
                int lmin = N, lmax = -1;
                for (int l = 0; l < N; ++l)
                    if (rv(fc, m, l) != 0.0) { lmin = std::min(lmin, l); lmax = std::max(lmax, l); }
                if (lmax < 0) continue;
                std::fprintf(f, "    if (LO <= %d && %d < HI) { const R x = g[%d * stride];", lmax, lmin, m);
                for (int l = 0; l < N; ++l) {
                    double c = rv(fc, m, l);
                    if (c == 0.0) continue;
                    std::fprintf(f, " if (LO <= %d && %d < HI) acc[%d] = fmaa(", l, l, l);
                    lit(f, c);
                    std::fprintf(f, ", x, acc[%d]);", l);
                }
                std::fprintf(f, " }\n");
            }
            std::fprintf(f, "  }\n};\n");
        }
        for (int a = 0; a < 3; ++a) {
            std::fprintf(f, "template <> struct DerivOp<%d, %d> {\n  template <typename R, int LO = 0, int HI = %d>\n"
                            "  __device__ static __forceinline__ void apply(const R* v, int stride, R sign, R* acc) {\n",
                         p, a, N);
            for (int m = 0; m < N; ++m) {
                int lmin = N, lmax = -1;
                for (int l = 0; l < N; ++l)
                    if (sv(a, l, m) != 0.0) { lmin = std::min(lmin, l); lmax = std::max(lmax, l); }
                if (lmax < 0) continue;
                std::fprintf(f, "    if (LO <= %d && %d < HI) { const R x = sign * v[%d * stride];", lmax, lmin, m);
                for (int l = 0; l < N; ++l) {
                    double c = sv(a, l, m);
                    if (c == 0.0) continue;
                    ++nnzS;
                    std::fprintf(f, " if (LO <= %d && %d < HI) acc[%d] = fmaa(", l, l, l);
                    lit(f, c);
                    std::fprintf(f, ", x, acc[%d]);", l);
                }
                std::fprintf(f, " }\n");
            }
            std::fprintf(f, "  }\n};\n");
        }
        // transposed derivative (adjoint): acc[m] += sign sum_l S_a[l][m] v[l], rows m in [LO, HI)
        for (int a = 0; a < 3; ++a) {
            std::fprintf(f, "template <> struct DerivTOp<%d, %d> {\n  template <typename R, int LO = 0, int HI = %d>\n"
                            "  __device__ static __forceinline__ void apply(const R* v, int stride, R sign, R* acc) {\n",
                         p, a, N);
            for (int l = 0; l < N; ++l) {
                int mmin = N, mmax = -1;
                for (int m = 0; m < N; ++m)
                    if (sv(a, l, m) != 0.0) { mmin = std::min(mmin, m); mmax = std::max(mmax, m); }
                if (mmax < 0) continue;
                std::fprintf(f, "    if (LO <= %d && %d < HI) { const R x = sign * v[%d * stride];", mmax, mmin, l);
                for (int m = 0; m < N; ++m) {
                    double c = sv(a, l, m);
                    if (c == 0.0) continue;
                    std::fprintf(f, " if (LO <= %d && %d < HI) acc[%d] = fmaa(", m, m, m);
                    lit(f, c);
                    std::fprintf(f, ", x, acc[%d]);", m);
                }
                std::fprintf(f, " }\n");
            }
            std::fprintf(f, "  }\n};\n");
        }
        std::fprintf(f, "template <> struct RefNnz<%d> { static constexpr int S = %d, R = %d; };\n",
                     p, nnzS, nnzR);
        std::fprintf(f, "static const double kRefS_p%d[%d] = {", p, 3 * N * N);
        for (size_t i = 0; i < S.size(); ++i) std::fprintf(f, "%s%.17g", i ? "," : "", S[i]);
        std::fprintf(f, "};\nstatic const double kRefR_p%d[%d] = {", p, 4 * NF * N);
        for (size_t i = 0; i < Rm.size(); ++i) std::fprintf(f, "%s%.17g", i ? "," : "", Rm[i]);
        std::fprintf(f, "};\n\n");
    }
    std::fprintf(f, "inline const double* ref_S_compiled(int p) {\n  switch (p) {\n");
    for (int p = 1; p <= PMAX; ++p) std::fprintf(f, "    case %d: return kRefS_p%d;\n", p, p);
    std::fprintf(f, "    default: return nullptr;\n  }\n}\n");
    std::fprintf(f, "inline const double* ref_R_compiled(int p) {\n  switch (p) {\n");
    for (int p = 1; p <= PMAX; ++p) std::fprintf(f, "    case %d: return kRefR_p%d;\n", p, p);
    std::fprintf(f, "    default: return nullptr;\n  }\n}\n\n}  // namespace dgm\n");
    std::fclose(f);
    return 0;
}
