"""Oracle for the filament-suspension hot path: plain, slow, FP64, CPU only.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import,
call, link or execute anything in this package. The library package
``paper_1903_12609_gb300`` never imports it and shares no code with it: the
CUDA path must stand or fall on its own kernels.

Modules:
  rpy      -- RPY mobility apply, a plain C double loop (Sec. 2.7.1) loaded
              through ctypes.
  filament -- quaternion algebra, the discrete Kirchhoff-rod forces and
              torques, the BDF2 / Lie-group residual, the block-diagonal
              approximate Jacobian of App. B.2, the limited-memory bad Broyden
              iteration (Algorithm 2) and the timestep driver, in numpy FP64.
"""
