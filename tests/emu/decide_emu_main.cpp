// Driver of the Krylov convergence decision (test support): bicg_decide on a
// control block, printing the status it sets, for the squared residual ratio,
// the launch's tolerance and the state's inner tolerance given.
//
// usage: decide_emu rr_over_bb tol2 tol2_in it maxit
//   prints the status (ST_*), then beta and rho[0]

int main(int argc, char** argv) {
    if (argc != 6) return 1;
    SliceCtl c{};
    c.bb = 4.0;
    c.it_cur = std::atoi(argv[4]);
    c.alpha = 0.5;
    c.omega = 0.25;
    c.rho[0] = 2.0;
    c.tol2_in = std::atof(argv[3]);
    const double rr = std::atof(argv[1]) * c.bb;
    bicg_decide(&c, 3.0, rr, 0.0, std::atof(argv[2]), std::atoi(argv[5]));
    std::printf("%d %.17g %.17g\n", c.status, c.beta, c.rho[0]);
    return 0;
}
