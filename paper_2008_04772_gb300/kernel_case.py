"""Single-kernel cases for profiling (the launches named in profiles/).

``python -m paper_2008_04772_gb300.kernel_case [bc|gemv|all]`` on the 5120-triangle
sphere (k = 5):
  bc    one dense FP32 assembly of S and C on the Buffa–Christiansen space
        (one bc_tile_kernel launch plus the FP64 singular-pair launch);
  gemv  an unpreconditioned FP32 solve capped at 3 GMRES iterations (the
        PMCHWT GEMV launches on the stored A blocks);
  all   both, in this order.
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
        op = cal.assemble(ctx, cal.OP_S | cal.OP_C, 5.0, bc, precision=cal.FP32)
        del op
    if which in ("all", "gemv"):
        cal.pmchwt_solve(ctx, mesh, 5.0, 3.17 + 0.01j, meshgen.plane_wave_x_along_z(),
                         opts=cal.solve_opts(precond="none", precision=cal.FP32, maxit=3, refine=0),
                         allow_not_converged=True)
    print("kernel_case done:", which)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "all")
