"""GB300-native batched Parareal projection stepper (placeholder, binding follows)."""
