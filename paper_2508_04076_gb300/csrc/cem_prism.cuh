// Division of a triangular prism into three tetrahedra (Sec. 3: the prism that
// remains of a split element is divided into three tetrahedra).
//
// The prism has the triangle A0 A1 A2 below B0 B1 B2, with rails Ai - Bi.  Each
// quadrilateral face is cut along the diagonal through its vertex with the
// smallest id, so two elements sharing a quadrilateral (neighbours split by the
// same crack) cut it alike and the sub-element mesh stays conforming.  With the
// prism turned so that its smallest vertex is v1 (v1 v2 v3 one triangle, v4 v5 v6
// the other, rails v1-v4, v2-v5, v3-v6), the faces through v1 take the diagonals
// v1-v5 and v1-v6, and the third face v2 v3 v6 v5 takes v2-v6 when
// min(v2, v6) < min(v3, v5), else v3-v5; each case has one division into three
// tetrahedra.  Orientation is left to the caller.
//
// A and B hold the vertices as stored; Ae and Be their creation ids, which fix
// the diagonals (so the division does not depend on storage order).  Written for
// both host and device so that a host test can check it against its definition.
#pragma once

#ifndef __CUDACC__
#define CEM_HD inline
#else
#define CEM_HD __host__ __device__ __forceinline__
#endif

CEM_HD void cem_prism_division(const int A[3], const int B[3], const int Ae[3], const int Be[3], int out[3][4]) {
    int i = 0, best = Ae[0];
    for (int q = 1; q < 6; ++q) {
        const int e = q < 3 ? Ae[q] : Be[q - 3];
        if (e < best) {
            best = e;
            i = q;
        }
    }
    const int j = i % 3;
    const int* lo = i < 3 ? A : B;
    const int* hi = i < 3 ? B : A;
    const int* loe = i < 3 ? Ae : Be;
    const int* hie = i < 3 ? Be : Ae;
    const int j1 = (j + 1) % 3, j2 = (j + 2) % 3;
    const int v1 = lo[j], v2 = lo[j1], v3 = lo[j2], v4 = hi[j], v5 = hi[j1], v6 = hi[j2];
    const int e2 = loe[j1], e3 = loe[j2], e5 = hie[j1], e6 = hie[j2];
    const int m26 = e2 < e6 ? e2 : e6, m35 = e3 < e5 ? e3 : e5;
    if (m26 < m35) {
        const int t[3][4] = {{v1, v2, v3, v6}, {v1, v2, v6, v5}, {v1, v5, v6, v4}};
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 4; ++c) out[r][c] = t[r][c];
    } else {
        const int t[3][4] = {{v1, v2, v3, v5}, {v1, v5, v3, v6}, {v1, v5, v6, v4}};
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 4; ++c) out[r][c] = t[r][c];
    }
}

#undef CEM_HD
