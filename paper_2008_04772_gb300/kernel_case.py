"""Single-kernel cases for profiling (the launches named in profiles/).

``python -m paper_2008_04772_gb300.kernel_case [bc|gemv|all]`` on the 5120-triangle
sphere (k = 5), with the benchmark's regular rules (near / medium / far classes at
the paper's default orders 4, 3, 2):
  bc    one dense FP32 assembly of S and C on the Buffa–Christiansen space
        (one bc_tile_kernel launch plus the FP64 singular-pair launch);
  gemv  an unpreconditioned FP32 solve capped at 3 GMRES iterations (the
        PMCHWT GEMV launches on the stored A blocks);
  gemm  the tensor-core product of the stored 7680 x 7680 complex64 S block
        with 32 vectors (cal_matvec, 3xTF32 on tcgen05);
  free  three FP32 GMRES iterations with the matrix-free PMCHWT operator (A8);
  solve one complete solve of the benchmark workload (FP32 bulk, full D, tol 1e-5),
        for the launch list;
  multi one FP32 solve of 32 incident directions with the near-field reduced
        preconditioner Di (chi = 2h): the multi-vector CSR product, the 64-system
        Gram BiCGStab and the double-float float64 refinement product;
  all   bc, gemv, gemm and free, in this order.
"""
import sys

from paper_2008_04772_gb300 import build, cal, meshgen


def main(which: str = "all") -> None:
    build.build()
    ctx = cal.Context(0)
    m = meshgen.icosphere(4)
    mesh = cal.Mesh(ctx, m.verts, m.tris, m.domain)
    if which in ("all", "bc"):
        bc = cal.Space(mesh, cal.BC)
        op = cal.assemble(ctx, cal.OP_S | cal.OP_C, 5.0, bc, q_regular=0, precision=cal.FP32)
        del op
    if which in ("all", "gemm"):
        import numpy as np
        import torch
        rwg = cal.Space(mesh, cal.RWG)
        op = cal.assemble(ctx, cal.OP_S, 5.0, rwg, precision=cal.FP32)
        n = op.info().cols
        x = torch.randn((32, 2 * n), dtype=torch.float32, device="cuda")
        y = torch.zeros((32, 2 * n), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        for _ in range(3):
            op.matvec(cal.OP_S, x.data_ptr(), y.data_ptr(), nrhs=32)
        torch.cuda.synchronize()
        del op, np
    if which in ("all", "free"):
        # three FP32 GMRES iterations with the matrix-free operator (float32 vectors)
        cal.pmchwt_solve(ctx, mesh, 5.0, 3.17 + 0.01j, meshgen.plane_wave_x_along_z(),
                         opts=cal.solve_opts(precond="none", precision=cal.FP32, maxit=3, refine=0,
                                             matrix_free=1, q_regular_A=0),
                         allow_not_converged=True)
    if which in ("all", "gemv"):
        cal.pmchwt_solve(ctx, mesh, 5.0, 3.17 + 0.01j, meshgen.plane_wave_x_along_z(),
                         opts=cal.solve_opts(precond="none", precision=cal.FP32, maxit=3, refine=0),
                         allow_not_converged=True)
    if which == "multi":
        d = meshgen.fibonacci_directions(32)
        import numpy as np
        inc = np.concatenate([d, meshgen.perpendicular_polarisation(d)], 1)
        cal.pmchwt_solve(ctx, mesh, 5.0, 3.17 + 0.01j, inc,
                         opts=cal.solve_opts(precond="Di", near_cutoff_P=2.0, precision=cal.FP32, tol=1e-5,
                                             q_regular_A=0, q_regular_P=0))
    if which == "solve":
        sol = cal.pmchwt_solve(ctx, mesh, 5.0, 3.17 + 0.01j, meshgen.plane_wave_x_along_z(),
                               opts=cal.solve_opts(precond="D", precision=cal.FP32, tol=1e-5, q_regular_A=0,
                                                   q_regular_P=0))
        sol.far_field(meshgen.sphere_cut_directions(181))
    print("kernel_case done:", which)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "all")
