/*
 * A plain C99 program against include/glbe.h and include/glbe2d.h: it shows
 * that the headers are C (not C++) and that the host-side entry points of
 * libglbe.so (defaults, validation, workspace sizing, error messages) work
 * from C with no GPU.  Prints one line per check; exits non-zero on the first
 * failure.  Built and run by tests/test_c_abi.py.
 */
#include <stdio.h>
#include <string.h>

#include "glbe.h"
#include "glbe2d.h"

static int failures = 0;

static void check(int ok, const char* what)
{
    printf("%s %s\n", ok ? "ok" : "FAIL", what);
    if (!ok) ++failures;
}

int main(void)
{
    glbe_params p;
    size_t bytes = 0, b16 = 0, bm = 0, pb = 0, ib = 0;

    glbe_struct_sizes(&pb, &ib);
    check(pb == sizeof(glbe_params) && ib == sizeof(glbe_residual_info), "struct sizes agree with the library");

    glbe_params_default(&p);
    check(p.rho0 == 1.0 && p.gamma == 1.0 && p.storage == GLBE_F32, "defaults: rho0 = 1, gamma = 1, F32");
    p.nx = 16;
    p.ny = 12;
    p.nz = 10;
    p.nu = 0.05;
    p.wall_lo[1] = p.wall_hi[1] = 1;
    check(glbe_workspace_bytes(&p, &bytes) == GLBE_OK, "workspace bytes of a walled duct");
    check(bytes >= (size_t)2 * 19 * 16 * 12 * 10 * sizeof(float), "workspace holds two FP32 population buffers");

    p.storage = GLBE_BF16;
    check(glbe_workspace_bytes(&p, &b16) == GLBE_OK && b16 < bytes, "BF16 storage needs less");
    p.storage = GLBE_F32;
    p.induction = 1;
    p.gamma_m = 0.5;
    p.eta = 0.01;
    p.chi = 0.1;
    p.mu = 1.0;
    check(glbe_workspace_bytes(&p, &bm) == GLBE_OK && bm > bytes, "the induction lattice needs more");

    p.gamma = 1.5;
    check(glbe_workspace_bytes(&p, &bytes) == GLBE_ERR_ARG, "gamma > 1 is rejected");
    check(glbe_last_error() != NULL && strlen(glbe_last_error()) > 0, "with a message");
    p.gamma = 0.5;
    p.nx = 0;
    check(glbe_workspace_bytes(&p, &bytes) == GLBE_ERR_ARG, "an empty grid is rejected");
    p.nx = 16;

    {
        size_t ab = 0, au = 0;
        check(glbe_adjoint_workspace_bytes(&p, 0, 1, &ab) == GLBE_OK && ab > 0, "steady adjoint workspace");
        check(glbe_adjoint_workspace_bytes(&p, 200, 20, &au) == GLBE_OK && au > ab,
              "unrolled adjoint workspace holds its checkpoints");
        check(glbe_adjoint_workspace_bytes(&p, -1, 1, &ab) == GLBE_ERR_ARG, "negative nsteps is rejected");
    }
    {
        glbe_params d[2];
        size_t bb = 0;
        d[0] = p;
        d[1] = p;
        d[1].induction = 0;
        check(glbe_batch_workspace_bytes(d, 2, &bb) == GLBE_OK && bb > 0, "batch workspace of two ducts");
    }

    {
        glbe2d_params q;
        size_t w = 0;
        glbe2d_params_default(&q);
        check(q.rho0 == 1.0 && q.storage == GLBE_F32, "2D defaults");
        q.nx = 32;
        q.ny = 18;
        q.nu = 0.05;
        q.wall_lo[1] = q.wall_hi[1] = 1;
        check(glbe2d_workspace_bytes(&q, &w) == GLBE_OK && w >= (size_t)2 * 9 * 32 * 18 * sizeof(float),
              "2D workspace bytes");
        q.variant = 7;
        check(glbe2d_workspace_bytes(&q, &w) == GLBE_ERR_ARG, "2D: an unknown variant is rejected");
    }

    check(glbe_step_n(NULL, 1) == GLBE_ERR_ARG, "a NULL context is rejected before any CUDA call");
    glbe_destroy(NULL);
    glbe2d_destroy(NULL);

    printf("%d failure(s)\n", failures);
    return failures ? 1 : 0;
}
