"""The boundary as a C program sees it, without a GPU: every public header
compiles as strict C99, and a C program linked against the in-tree library
calls the host-only entry points (version, planning, the pair schedule) and
gets what the Python binding gets."""
import glob
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2505_02438_gb300 import build, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INC = os.path.join(ROOT, "include")

pytestmark = pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")

PROGRAM = r"""
#include <stdio.h>
#include <stdlib.h>
#include "soptx.h"
#include "soptx_serve.h"
#include "soptx_solve.h"
#include "soptx_opt.h"

int main(void)
{
    /* 3 x 2 unit squares, each split into two triangles along (i,j)-(i+1,j+1) */
    enum { NX = 3, NY = 2 };
    double coords[(NX + 1) * (NY + 1) * 2];
    int32_t cells[NX * NY * 2 * 3];
    for (int j = 0; j <= NY; j++)
        for (int i = 0; i <= NX; i++) {
            coords[2 * (j * (NX + 1) + i)] = i;
            coords[2 * (j * (NX + 1) + i) + 1] = j;
        }
    int c = 0;
    for (int j = 0; j < NY; j++)
        for (int i = 0; i < NX; i++) {
            int v0 = j * (NX + 1) + i, v1 = v0 + 1, v2 = v0 + NX + 1, v3 = v2 + 1;
            cells[c++] = v0; cells[c++] = v1; cells[c++] = v3;
            cells[c++] = v0; cells[c++] = v3; cells[c++] = v2;
        }
    int64_t ndof = 0, nnz = 0;
    int32_t nb = 0;
    soptx_path path;
    if (soptx_host_plan(2, SOPTX_TRI, 3, (NX + 1) * (NY + 1), coords, NX * NY * 2, cells, &ndof, &nnz, &nb, &path,
                        NULL, NULL, NULL) != SOPTX_OK)
        return 1;
    int64_t *indptr = malloc(sizeof(int64_t) * (size_t)(ndof + 1));
    int32_t *indices = malloc(sizeof(int32_t) * (size_t)nnz);
    if (soptx_host_plan(2, SOPTX_TRI, 3, (NX + 1) * (NY + 1), coords, NX * NY * 2, cells, NULL, NULL, NULL, NULL,
                        indptr, indices, NULL) != SOPTX_OK)
        return 2;
    long long sum = 0;
    for (int64_t q = 0; q < nnz; q++) sum += indices[q];
    int64_t tiles = 0, recs = 0;
    if (soptx_host_pair_tables(2, SOPTX_TRI, 3, (NX + 1) * (NY + 1), coords, NX * NY * 2, cells, 0, &tiles, &recs,
                               NULL, NULL, NULL, NULL, NULL, NULL) != SOPTX_OK)
        return 3;
    /* a malformed call fails with EINVAL and a message, it does not abort */
    if (soptx_host_plan(2, SOPTX_TRI, 4, 1, coords, 0, NULL, &ndof, NULL, NULL, NULL, NULL, NULL, NULL) != SOPTX_EINVAL
        || soptx_last_error()[0] == '\0')
        return 4;
    printf("%s\n%lld %lld %d %d %lld %lld %lld\n", soptx_version(), (long long)ndof, (long long)nnz, (int)nb,
           (int)path, sum, (long long)tiles, (long long)recs);
    free(indptr);
    free(indices);
    return 0;
}
"""


@pytest.mark.parametrize("header", sorted(os.path.basename(h) for h in glob.glob(os.path.join(INC, "*.h"))))
def test_header_is_strict_c99(header, tmp_path):
    src = tmp_path / "h.c"
    src.write_text('#include "%s"\nint main(void) { return 0; }\n' % header)
    subprocess.run(["gcc", "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror", "-fsyntax-only", "-I", INC,
                    str(src)], check=True, capture_output=True, text=True)


def test_c_program_calls_the_host_entry_points(tmp_path):
    build.build_library()
    from paper_2505_02438_gb300 import _native
    from paper_2505_02438_gb300.api import host_pair_tables, host_plan
    lib = _native.LIB_PATH
    src, exe = tmp_path / "consumer.c", tmp_path / "consumer"
    src.write_text(PROGRAM)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", INC, str(src), "-o", str(exe), lib,
                    "-Wl,-rpath," + os.path.dirname(lib)], check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    assert "sm_103a" in out[0]
    ndof, nnz, nb, path, isum, tiles, recs = (int(x) for x in out[1].split())
    coords, cells = W.structured_quad(3, 2)
    coords = coords.astype(np.float64)
    tri = np.concatenate([cells[:, [0, 1, 3]], cells[:, [0, 3, 2]]], axis=1).reshape(-1, 3)
    pl = host_plan("tri", 3, coords, tri)
    T = host_pair_tables("tri", 3, coords, tri)
    assert (ndof, nnz, nb) == (pl["ndof"], pl["nnz"], pl["nb"]) and isum == int(pl["indices"].sum())
    assert (tiles, recs) == (T["n_tiles"], len(T["record_cell"]))
