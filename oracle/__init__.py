"""Plain, slow FP64 CPU oracle of the MPS lattice Boltzmann method
(Gross, Mounzer, Wawrzyniak, Winter, Adams: "Tensor Network Lattice Boltzmann
Method for Data-Compressed Fluid Simulations").

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call, link or
execute this package: only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline leg use it.  It shares no code, tables or helpers with the CUDA library
under paper_2512_07615_gb300/.

Modules
  quantics  scale-ordered binary site encoding (Sec. 2.4, Eq. scale_ordering)
  mps       MPS algebra: TT-SVD (Eq. svd-comp), rounding (Eq. svd-move),
            addition (Eq. add), exact product (Eq. mul), MPO application
            (Eq. applympo), compressed product by single-site fit (Sec. 2.3)
  mpo       cyclic and non-cyclic shift MPOs (Sec. 2.5, Eq. recursive)
  lattice   D3Q19 / D3Q15 velocity sets (Sec. 3.1)
  lbm_dense full-grid BGK LBM with exact or Taylor 1/rho (Sec. 3, App. A)
  mps_lbm   the MPS-LBM time step (Sec. 3.2)
  metrics   relative l2 error and compression ratio (Sec. 3.2, Eq. for NVPS)

Precision: float64 throughout; numpy.linalg QR/SVD serve as library steps.
Parity status per function is stated in each module header.
"""
