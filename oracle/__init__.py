"""Plain FP64 CPU oracle of the Palabos Turret time step (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may use it;
the product package never imports it.
"""
